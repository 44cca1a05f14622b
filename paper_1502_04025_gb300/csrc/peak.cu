// Arithmetic peaks of the device, measured: a fused multiply-add chain kernel
// in FP64 or FP32 (the denominators of the rooflines of the ALU-bound steps:
// the FP64 operator and vector algebra of the outer solver, and the FP32
// Schwarz sweeps).  Not part of the method; a measurement service.
//
// Every thread runs kChains independent chains x <- x * a + b (a just below
// one, so the values stay finite), enough independent work per warp to cover
// the pipeline latency; the grid fills every SM several times over.  Flops
// are counted as 2 per FMA.  The result is written only under a condition the
// compiler cannot decide, so the chains are not removed.
#include "internal.h"

namespace qdd {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;

__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }
__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chain(T a, T b, int iters, T *out)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fma_t(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static qdd_status run_chain(int nsm, int iters, T *out, float *ms)
{
    cudaEvent_t e0, e1;
    QDD_CUDA(cudaEventCreate(&e0));
    QDD_CUDA(cudaEventCreate(&e1));
    QDD_CUDA(cudaEventRecord(e0, 0));
    k_fma_chain<T><<<nsm * kPeakBlocksPerSM, kPeakThreads>>>((T)0.9999999, (T)1e-7, iters, out);
    QDD_CUDA(cudaGetLastError());
    QDD_CUDA(cudaEventRecord(e1, 0));
    QDD_CUDA(cudaEventSynchronize(e1));
    QDD_CUDA(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return QDD_OK;
}

}  // namespace qdd

extern "C" qdd_status qdd_measure_fma_peak(int device, int fp64, double target_ms, double *tflops, double *ms_out)
{
    using namespace qdd;
    clear_error();
    if (!tflops || !(target_ms > 0) || target_ms > 10000) {
        set_error("tflops must be non-null and target_ms in (0, 10000]");
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaSetDevice(device));
    int nsm = 0;
    QDD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    const size_t nthreads = (size_t)nsm * kPeakBlocksPerSM * kPeakThreads;
    void *out = nullptr;
    QDD_CUDA(cudaMalloc(&out, nthreads * 8));
    qdd_status st = QDD_OK;
    float ms = 0;
    // calibrate the iteration count on a short run, then time one run of
    // about target_ms (the first short run also warms the clocks up)
    int iters = 256;
    for (int pass = 0; pass < 3 && st == QDD_OK; pass++) {
        st = fp64 ? run_chain<double>(nsm, iters, (double *)out, &ms) : run_chain<float>(nsm, iters, (float *)out, &ms);
        if (st != QDD_OK) break;
        if (pass < 2) {
            double scale = target_ms / (ms > 1e-3 ? ms : 1e-3);
            double next = iters * scale;
            iters = (int)(next < 1 ? 1 : (next > 2e9 ? 2e9 : next));
        }
    }
    cudaFree(out);
    if (st != QDD_OK) return st;
    const double flop = 2.0 * 8.0 * kChains * (double)iters * (double)nthreads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return QDD_OK;
}
