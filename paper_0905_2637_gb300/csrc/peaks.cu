// peaks.cu -- microbenchmarks of the pipes the kernels are bound by, so that
// roofline fractions can be quoted against this GPU's measured rates rather
// than only nominal ones: FP32 FFMA, FP64 DFMA, the special-function unit
// (rcp, ex2) and dense TF32 MMA on the 5th-generation tensor cores.
//
// Each SIMT kernel runs independent dependency chains (enough per thread to
// cover the pipe latency) over every SM, and writes one value per thread so
// that nothing is optimised away.  The TF32 kernel has one CTA per SM issue
// back-to-back M = 128, N = 256, K = 8 MMAs into one TMEM accumulator from
// operands in shared memory; its only wait is bounded.
#include <algorithm>

#include "../../include/petfmm.h"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace petfmm {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float b, float c, int iters,
                                                          float *out) {
    float a[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) a[i] = float(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(double b, double c, int iters,
                                                          double *out) {
    double a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = double(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = fma(a[i], b, c);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a[0] + a[1] + a[2] + a[3];
}

// mode 0: a <- rcp(a / 2 + 3/4) (stays in [4/7, 1] for a start in [1, 2]; one
// FFMA per rcp, so that no two consecutive rcp could be folded);
// mode 1: a <- ex2(-a) (stays in [1/2, 1] for a start in [0, 1]).
__global__ void __launch_bounds__(PK_THREADS) k_peak_mufu(int mode, int iters, float *out) {
    float a[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) a[i] = 1.0f + float((threadIdx.x + i) & 7) * 0.125f;
    if (mode == 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
#pragma unroll
                for (int i = 0; i < PK_CHAINS; ++i)
                    asm volatile("{\n.reg .f32 t;\nfma.rn.f32 t, %0, 0f3F000000, 0f3F400000;\n"
                                 "rcp.approx.ftz.f32 %0, t;\n}"
                                 : "+f"(a[i]));
            }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
#pragma unroll
                for (int i = 0; i < PK_CHAINS; ++i)
                    asm volatile("{\n.reg .f32 t;\nneg.f32 t, %0;\nex2.approx.ftz.f32 %0, t;\n}"
                                 : "+f"(a[i]));
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int PK_M = 128, PK_N = 256, PK_K = 8;

__global__ void __launch_bounds__(128, 1) k_peak_tf32(int nmma, long long spin_limit, int *status) {
    __shared__ __align__(1024) float A[PK_M * PK_K];
    __shared__ __align__(1024) float B[PK_N * PK_K];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    // K-major, no swizzle: [k group of 4][row][4 values]
    for (int i = tid; i < PK_M * PK_K; i += 128) A[i] = 1.0f / float(1 + (i & 63));
    for (int i = tid; i < PK_N * PK_K; i += 128) B[i] = 1.0f / float(1 + (i & 31));
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tslot)),
                     "r"(PK_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // operands written by the generic proxy, read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(PK_N >> 3) << 17) |
                           (uint32_t(PK_M >> 4) << 24);
    if (tid == 0) {
        const uint64_t da = mma_desc(smem_addr(A), PK_M * 16, 128);
        const uint64_t db = mma_desc(smem_addr(B), PK_N * 16, 128);
        for (int i = 0; i < nmma; ++i) mma_tf32(tbase, da, db, idesc, i > 0 ? 1u : 0u);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
    }
    const bool ok = __syncthreads_and(mbar_wait(bar, 0, spin_limit) ? 1 : 0) != 0;
    if (!ok && tid == 0) atomicCAS(status, 0, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(uint32_t(PK_N)));
}

}  // namespace petfmm

using namespace petfmm;

namespace {

// Best of three timed launches after one warm-up; returns the seconds.
template <typename F>
bool time_best(cudaStream_t st, F launch, double *sec) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return false;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return false;
    }
    bool ok = true;
    launch();
    double best = 1e30;
    for (int r = 0; r < 3 && ok; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
        float ms = 0.f;
        if (ok) cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, double(ms) * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *sec = best;
    return ok && best > 0.0;
}

}  // namespace

int petfmm_measure_peaks(petfmm_peaks *out) {
    if (!out) return PETFMM_EINVAL;
    const int sms = device_sm_count();
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PETFMM_ECUDA;
    const int blocks = sms * 8;
    const size_t nthreads = size_t(blocks) * PK_THREADS;
    void *buf = nullptr;
    int *status = nullptr;
    int rc = PETFMM_OK;
    if (cudaMalloc(&buf, nthreads * sizeof(double)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&status), sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rc = PETFMM_ENOMEM;
    }
    double sec = 0.0;
    if (rc == PETFMM_OK) {
        const int it = 4096;
        if (!time_best(st, [&] {
                k_peak_ffma<<<blocks, PK_THREADS, 0, st>>>(0.999f, 1e-3f, it,
                                                           static_cast<float *>(buf));
            }, &sec))
            rc = PETFMM_ECUDA;
        else
            out->fp32_ops = double(nthreads) * it * 16 * PK_CHAINS / sec;
    }
    if (rc == PETFMM_OK) {
        const int it = 256;
        if (!time_best(st, [&] {
                k_peak_dfma<<<blocks, PK_THREADS, 0, st>>>(0.999, 1e-3, it,
                                                           static_cast<double *>(buf));
            }, &sec))
            rc = PETFMM_ECUDA;
        else
            out->fp64_ops = double(nthreads) * it * 16 * 4 / sec;
    }
    for (int mode = 0; mode < 2 && rc == PETFMM_OK; ++mode) {
        const int it = 512;
        if (!time_best(st, [&] {
                k_peak_mufu<<<blocks, PK_THREADS, 0, st>>>(mode, it, static_cast<float *>(buf));
            }, &sec))
            rc = PETFMM_ECUDA;
        else
            (mode == 0 ? out->mufu_rcp_ops : out->mufu_ex2_ops) =
                double(nthreads) * it * 16 * PK_CHAINS / sec;
    }
    if (rc == PETFMM_OK) {
        const int nmma = 8192;
        cudaMemsetAsync(status, 0, sizeof(int), st);
        if (!time_best(st, [&] {
                k_peak_tf32<<<sms, 128, 0, st>>>(nmma, 1LL << 26, status);
            }, &sec)) {
            rc = PETFMM_ECUDA;
        } else {
            int h = 0;
            cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost);
            if (h) rc = PETFMM_ETIMEOUT;
            out->tf32_flops = double(sms) * nmma * 2.0 * PK_M * PK_N * PK_K / sec;
        }
    }
    cudaFree(buf);
    cudaFree(status);
    cudaStreamDestroy(st);
    out->sms = sms;
    return rc;
}
