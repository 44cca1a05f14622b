// FP64 complex vector algebra of the outer flexible GMRES (arXiv:1502.04025,
// Sec. 3.1: the outer solver is flexible GMRES).  Gram-Schmidt, norms,
// basis updates and the solution update run in FP64 on the device.
//
// Vectors are flat arrays of complex FP64 (double2); the lattice layout does
// not matter here.  All reductions are two-level and deterministic: a fixed
// number of blocks (a multiple of the SM count) writes per-block partials,
// and the last block to finish (a counter in the scratch buffer) sums them in
// block order; the allocation-free entry point sums them in a separate
// launch instead.  Fused forms read each vector once: the multi-dot reads w
// once for all basis vectors, the multi-axpy writes w once and returns its
// new norm.
#include <mutex>
#include <type_traits>

#include "internal.h"

namespace qdd {

constexpr int kBT = 256;       // threads per block
constexpr int kNV = 16;        // basis vectors per pass

int blas_blocks(const Ctx *ctx, int64_t n)
{
    int64_t want = (n + kBT - 1) / kBT;
    int64_t cap = 2LL * (ctx->nsm > 0 ? ctx->nsm : 148);
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

// per-block partials of up to 2 blocks per SM, then one slot whose first
// word counts the blocks that have finished (zero between launches)
size_t blas_scratch_elems(const Ctx *ctx) { return (size_t)2 * (ctx->nsm > 0 ? ctx->nsm : 148) * kNV + 1; }

static unsigned *scratch_counter(const Ctx *ctx, double2 *scratch)
{
    return (unsigned *)(scratch + blas_scratch_elems(ctx) - 1);
}

qdd_status blas_scratch_ensure(Ctx *ctx, DevMem &m)
{
    const size_t bytes = blas_scratch_elems(ctx) * sizeof(double2);
    if (m.p && m.bytes >= bytes) return QDD_OK;
    QDD_TRY(m.alloc(ctx, bytes));
    QDD_CUDA(cudaMemset(scratch_counter(ctx, m.as<double2>()), 0, sizeof(unsigned)));
    QDD_CUDA(cudaDeviceSynchronize());
    return QDD_OK;
}

__device__ __forceinline__ double2 dsum2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// sum of NV double2 over the block; result valid in threads 0..NV-1 via sm
template <int NV>
__device__ __forceinline__ void block_reduce(double2 *acc, double2 *sm /* [kBT/32][NV] */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
            acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
        }
        if (lane == 0) sm[w * NV + j] = acc[j];
    }
    __syncthreads();
}

// The last block to finish sums every block's partials (stride `stride`,
// nv values each) in block order, with the same arithmetic as
// k_reduce_final, writes out[0..nv) and resets the counter.  Called by all
// threads after the block's own partials are written.
template <int NV>
__device__ __forceinline__ void last_block_final(const double2 *part, int stride, int nv, unsigned *count,
                                                 double2 *out, double2 *sm /* [kBT/32][NV] */)
{
    __shared__ bool last;
    __threadfence();  // this block's partials before its count
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 acc[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) acc[j] = make_double2(0, 0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kBT)
#pragma unroll
        for (int j = 0; j < NV; j++)
            if (j < nv) acc[j] = dsum2(acc[j], __ldcg(part + (int64_t)b * stride + j));
    block_reduce<NV>(acc, sm);
    if (threadIdx.x < nv) {
        double2 t = make_double2(0, 0);
        for (int ww = 0; ww < kBT / 32; ww++) t = dsum2(t, sm[ww * NV + threadIdx.x]);
        out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *count = 0;
}

// count != NULL: the last block also writes the final sums to out
template <int NV>
__global__ void __launch_bounds__(kBT) k_cdot_partial(const double2 *__restrict__ v, int nvec, int64_t ld,
                                                      const double2 *__restrict__ w, int64_t n, double2 *part,
                                                      unsigned *count = nullptr, double2 *out = nullptr)
{
    __shared__ double2 sm[(kBT / 32) * NV];
    double2 acc[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) acc[j] = make_double2(0, 0);
    for (int64_t k = (int64_t)blockIdx.x * kBT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kBT) {
        double2 b = __ldg(w + k);
#pragma unroll
        for (int j = 0; j < NV; j++)
            if (j < nvec) {
                double2 a = __ldg(v + j * ld + k);
                acc[j].x = fma(a.x, b.x, acc[j].x);
                acc[j].x = fma(a.y, b.y, acc[j].x);
                acc[j].y = fma(a.x, b.y, acc[j].y);
                acc[j].y = fma(-a.y, b.x, acc[j].y);
            }
    }
    block_reduce<NV>(acc, sm);
    if (threadIdx.x < NV) {
        double2 s = make_double2(0, 0);
        for (int ww = 0; ww < kBT / 32; ww++) s = dsum2(s, sm[ww * NV + threadIdx.x]);
        part[(int64_t)blockIdx.x * kNV + threadIdx.x] = s;
    }
    if (count) {
        __syncthreads();  // sm is reused
        last_block_final<NV>(part, kNV, nvec, count, out, sm);
    }
}

// out[j] = sum over blocks of part[b*stride + j], j < nvec; one block per j
__global__ void __launch_bounds__(kBT) k_reduce_final(const double2 *part, int nblk, int stride, double2 *out,
                                                      int sqrt_x)
{
    __shared__ double2 sm[kBT / 32];
    const int j = blockIdx.x;
    double2 s = make_double2(0, 0);
    for (int b = threadIdx.x; b < nblk; b += kBT) s = dsum2(s, part[(int64_t)b * stride + j]);
    double2 acc[1] = {s};
    block_reduce<1>(acc, sm);
    if (threadIdx.x == 0) {
        double2 t = make_double2(0, 0);
        for (int ww = 0; ww < kBT / 32; ww++) t = dsum2(t, sm[ww]);
        out[j] = t;
    }
}

// w -= sum_j coef[j] v_j (j < nvec); optional per-block partial of |w|^2
template <int NV>
__global__ void __launch_bounds__(kBT) k_caxpy_norm(const double2 *__restrict__ v, int nvec, int64_t ld,
                                                    const double2 *__restrict__ coef, double2 *w, int64_t n,
                                                    double2 *part, unsigned *count, double2 *norm2_out)
{
    __shared__ double2 sm[kBT / 32];
    double2 c[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) c[j] = j < nvec ? coef[j] : make_double2(0, 0);
    double nrm = 0;
    for (int64_t k = (int64_t)blockIdx.x * kBT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kBT) {
        double2 b = w[k];
#pragma unroll
        for (int j = 0; j < NV; j++)
            if (j < nvec) {
                double2 a = __ldg(v + j * ld + k);
                b.x = fma(-c[j].x, a.x, b.x);
                b.x = fma(c[j].y, a.y, b.x);
                b.y = fma(-c[j].x, a.y, b.y);
                b.y = fma(-c[j].y, a.x, b.y);
            }
        if (nvec > 0) w[k] = b;
        nrm = fma(b.x, b.x, nrm);
        nrm = fma(b.y, b.y, nrm);
    }
    if (part) {
        double2 acc[1] = {make_double2(nrm, 0)};
        block_reduce<1>(acc, sm);
        if (threadIdx.x == 0) {
            double2 t = make_double2(0, 0);
            for (int ww = 0; ww < kBT / 32; ww++) t = dsum2(t, sm[ww]);
            part[blockIdx.x] = t;
        }
        __syncthreads();  // sm is reused
        last_block_final<1>(part, 1, 1, count, norm2_out, sm);
    }
}

// out = w / sqrt(norm2[0]) (out may alias w); out32 (optional) gets the same
// vector rounded to FP32
__global__ void k_scale_by_norm(const double2 *w, int64_t n, const double2 *norm2, double2 *out, float2 *out32)
{
    // once per block: FP64 square root and division are long sequences on
    // the FP64 pipe
    __shared__ double fs;
    if (threadIdx.x == 0) {
        double nn = norm2[0].x;
        fs = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    const double f = fs;
    for (int64_t k = (int64_t)blockIdx.x * kBT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kBT) {
        double2 a = w[k];
        a = make_double2(a.x * f, a.y * f);
        out[k] = a;
        if (out32) out32[k] = make_float2((float)a.x, (float)a.y);
    }
}

// x += sum_j coef[j] z_j, z in FP64 or FP32
template <typename T2>
__global__ void __launch_bounds__(kBT) k_axpy_multi(const T2 *__restrict__ z, int nvec, int64_t ld,
                                                    const double2 *__restrict__ coef, double2 *x, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * kBT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kBT) {
        double2 b = x[k];
        for (int j = 0; j < nvec; j++) {
            T2 a = z[j * ld + k];
            double2 cj = coef[j];
            double ax = (double)a.x, ay = (double)a.y;
            b.x = fma(cj.x, ax, b.x);
            b.x = fma(-cj.y, ay, b.x);
            b.y = fma(cj.x, ay, b.y);
            b.y = fma(cj.y, ax, b.y);
        }
        x[k] = b;
    }
}

// Basis recombination of a deflated restart: out_c (+)= sum_i src_i P[i][c]
// for the NC columns c0..c0+NC-1 of P (row-major, ldp columns), src in FP64
// or FP32, out in FP64.
template <typename T2, int NC>
__global__ void __launch_bounds__(kBT) k_combine(const T2 *__restrict__ src, int nsrc, int64_t ld,
                                                 const double2 *__restrict__ P, int ldp, int c0, double2 *out,
                                                 int64_t ldo, int64_t n, int accumulate)
{
    for (int64_t k = (int64_t)blockIdx.x * kBT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kBT) {
        double2 acc[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) acc[c] = accumulate ? out[(int64_t)c * ldo + k] : make_double2(0, 0);
        for (int i = 0; i < nsrc; i++) {
            T2 a = src[i * ld + k];
            double ax = (double)a.x, ay = (double)a.y;
#pragma unroll
            for (int c = 0; c < NC; c++) {
                double2 p = __ldg(P + (int64_t)i * ldp + c0 + c);
                acc[c].x = fma(p.x, ax, acc[c].x);
                acc[c].x = fma(-p.y, ay, acc[c].x);
                acc[c].y = fma(p.x, ay, acc[c].y);
                acc[c].y = fma(p.y, ax, acc[c].y);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; c++) out[(int64_t)c * ldo + k] = acc[c];
    }
}

// ------------------------------------------------------------- launchers

// Call f with std::integral_constant<int, NV> for NV = nv (1..kNV): kernels
// are instantiated for exactly the number of vectors they handle, because
// predicated-off iterations of a wider unrolled loop would still occupy the
// FP64 pipe, the bottleneck of these kernels on this GPU.
template <typename F>
static void nv_dispatch(int nv, F &&f)
{
    switch (nv) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    case 10: f(std::integral_constant<int, 10>{}); break;
    case 11: f(std::integral_constant<int, 11>{}); break;
    case 12: f(std::integral_constant<int, 12>{}); break;
    case 13: f(std::integral_constant<int, 13>{}); break;
    case 14: f(std::integral_constant<int, 14>{}); break;
    case 15: f(std::integral_constant<int, 15>{}); break;
    default: f(std::integral_constant<int, 16>{}); break;
    }
}

qdd_status blas_cdot_multi(Ctx *ctx, const double2 *v, int nvec, int64_t ld, const double2 *w, int64_t n,
                           double2 *out, double2 *scratch, cudaStream_t s)
{
    if (nvec <= 0) return QDD_OK;
    const int nb = blas_blocks(ctx, n);
    for (int j0 = 0; j0 < nvec; j0 += kNV) {
        int nv = nvec - j0 < kNV ? nvec - j0 : kNV;
        ctx->timer.work(K_BLAS, 8.0 * nv * n, 16.0 * (nv + 1) * n);
        LaunchScope ls(ctx->timer, K_BLAS, s);
        nv_dispatch(nv, [&](auto c) {
            k_cdot_partial<decltype(c)::value><<<nb, kBT, 0, s>>>(v + j0 * ld, nv, ld, w, n, scratch,
                                                                  scratch_counter(ctx, scratch), out + j0);
        });
    }
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status blas_caxpy_multi_norm(Ctx *ctx, const double2 *v, int nvec, int64_t ld, const double2 *coef, double2 *w,
                                 int64_t n, double2 *norm2_out, double2 *scratch, cudaStream_t s)
{
    const int nb = blas_blocks(ctx, n);
    int j0 = 0;
    do {
        int nv = nvec - j0 < kNV ? nvec - j0 : kNV;
        bool last = j0 + nv >= nvec;
        // v read, w read and (when updated) written; |w|^2 on the last pass
        ctx->timer.work(K_BLAS, 8.0 * nv * n + ((last && norm2_out) ? 4.0 * n : 0.0),
                        16.0 * (nv + 1 + (nv > 0 ? 1 : 0)) * n);
        {
            LaunchScope ls(ctx->timer, K_BLAS, s);
            double2 *part = (last && norm2_out) ? scratch : nullptr;
            unsigned *cnt = scratch_counter(ctx, scratch);
            if (nv == 0)
                k_caxpy_norm<1><<<nb, kBT, 0, s>>>(v, 0, ld, coef, w, n, part, cnt, norm2_out);
            else
                nv_dispatch(nv, [&](auto c) {
                    k_caxpy_norm<decltype(c)::value><<<nb, kBT, 0, s>>>(v + j0 * ld, nv, ld, coef + j0, w, n, part,
                                                                        cnt, norm2_out);
                });
        }
        j0 += nv;
    } while (j0 < nvec);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status blas_norm2(Ctx *ctx, const double2 *w, int64_t n, double2 *out, double2 *scratch, cudaStream_t s)
{
    return blas_caxpy_multi_norm(ctx, nullptr, 0, 0, nullptr, (double2 *)w, n, out, scratch, s);
}

qdd_status blas_scale_by_norm(Ctx *ctx, const double2 *w, int64_t n, const double2 *norm2, double2 *out,
                              cudaStream_t s, float2 *out32)
{
    // one element per thread: a memory-bound pass needs every load in flight
    // at once (the reduction kernels' two blocks per SM keep too few)
    const int64_t nb = (n + kBT - 1) / kBT;
    ctx->timer.work(K_BLAS, 2.0 * n, (32.0 + (out32 ? 8.0 : 0.0)) * n);
    LaunchScope ls(ctx->timer, K_BLAS, s);
    k_scale_by_norm<<<(unsigned)(nb < (1LL << 30) ? nb : (1LL << 30)), kBT, 0, s>>>(w, n, norm2, out, out32);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status blas_combine(Ctx *ctx, const void *src, bool src_f32, int nsrc, int64_t ld, const double2 *P, int ldp,
                        int ncols, double2 *out, int64_t ldo, int64_t n, int accumulate, cudaStream_t s)
{
    if (nsrc <= 0 || ncols <= 0) return QDD_OK;
    const int nb = blas_blocks(ctx, n);
    for (int c0 = 0; c0 < ncols; c0 += kNV) {
        int nc = ncols - c0 < kNV ? ncols - c0 : kNV;
        ctx->timer.work(K_BLAS, 8.0 * nsrc * nc * n,
                        ((src_f32 ? 8.0 : 16.0) * nsrc + 16.0 * nc * (accumulate ? 2 : 1)) * n);
        LaunchScope ls(ctx->timer, K_BLAS, s);
        nv_dispatch(nc, [&](auto c) {
            if (src_f32)
                k_combine<float2, decltype(c)::value><<<nb, kBT, 0, s>>>((const float2 *)src, nsrc, ld, P, ldp, c0,
                                                                         out + (int64_t)c0 * ldo, ldo, n, accumulate);
            else
                k_combine<double2, decltype(c)::value><<<nb, kBT, 0, s>>>((const double2 *)src, nsrc, ld, P, ldp, c0,
                                                                          out + (int64_t)c0 * ldo, ldo, n,
                                                                          accumulate);
        });
    }
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status blas_axpy_multi(Ctx *ctx, const void *z, bool z_f32, int nvec, int64_t ld, const double2 *coef,
                           double2 *x, int64_t n, cudaStream_t s)
{
    if (nvec <= 0) return QDD_OK;
    ctx->timer.work(K_BLAS, 8.0 * nvec * n, ((z_f32 ? 8.0 : 16.0) * nvec + 32.0) * n);
    LaunchScope ls(ctx->timer, K_BLAS, s);
    if (z_f32)
        k_axpy_multi<float2><<<blas_blocks(ctx, n), kBT, 0, s>>>((const float2 *)z, nvec, ld, coef, x, n);
    else
        k_axpy_multi<double2><<<blas_blocks(ctx, n), kBT, 0, s>>>((const double2 *)z, nvec, ld, coef, x, n);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free multi-dot (qdd_cdot_multi_noalloc).
//
// The per-block partial sums live in a fixed device array that is part of the
// library image instead of in memory from cudaMalloc.  Host code may not use
// the array's name as a device pointer: it only stands in for the symbol, so
// the device address is looked up once per device with cudaGetSymbolAddress
// and passed to the kernels.  The array holds kNoAllocBlocks * kNV partials
// (128 KiB) on every GPU that loads the library, until the process exits.

constexpr int kNoAllocBlocks = 512;
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocBlocks * kNV];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double2 *g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_nsm[kMaxDevices] = {};

// Device address of the partials array on the current device, resolved on
// the first call for that device.
qdd_status noalloc_setup(int dev, double2 **ptr, int *nsm)
{
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d out of range for the allocation-free entry points", dev);
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the partial-sum array failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return QDD_ECUDA;
        }
        int sm = 0;
        e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            set_error("cudaDeviceGetAttribute failed on device %d: %s", dev, cudaGetErrorString(e));
            return QDD_ECUDA;
        }
        g_noalloc_nsm[dev] = sm;
        g_noalloc_ptr[dev] = (double2 *)p;
    }
    *ptr = g_noalloc_ptr[dev];
    *nsm = g_noalloc_nsm[dev];
    return QDD_OK;
}
}  // namespace

}  // namespace qdd

extern "C" qdd_status qdd_cdot_multi_noalloc(const double *v, int nvec, int64_t ld, const double *w, int64_t n,
                                             double *out, void *stream)
{
    using namespace qdd;
    clear_error();
    if (!v || !w || !out) {
        set_error("null pointer argument");
        return QDD_EINVAL;
    }
    if (nvec < 1 || nvec > 64) {
        set_error("nvec = %d outside 1..64", nvec);
        return QDD_EINVAL;
    }
    if (n < 1 || n > (int64_t(1) << 40) || ld < n) {
        set_error("vector length n = %lld (stride %lld) outside 1..2^40 or stride below n", (long long)n,
                  (long long)ld);
        return QDD_EINVAL;
    }
    int dev = 0;
    QDD_CUDA(cudaGetDevice(&dev));
    double2 *part = nullptr;
    int nsm = 0;
    QDD_TRY(noalloc_setup(dev, &part, &nsm));
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nb64 = (n + kBT - 1) / kBT;
    int64_t cap = 2LL * nsm;
    if (cap > kNoAllocBlocks) cap = kNoAllocBlocks;
    if (nb64 > cap) nb64 = cap;
    const int nb = (int)(nb64 < 1 ? 1 : nb64);
    const double2 *V2 = (const double2 *)v, *W2 = (const double2 *)w;
    double2 *O2 = (double2 *)out;
    // every block overwrites its own partials before the final sum reads them,
    // so nothing in the shared array has to start at zero
    for (int j0 = 0; j0 < nvec; j0 += kNV) {
        int nv = nvec - j0 < kNV ? nvec - j0 : kNV;
        nv_dispatch(nv, [&](auto c) {
            k_cdot_partial<decltype(c)::value><<<nb, kBT, 0, s>>>(V2 + j0 * ld, nv, ld, W2, n, part);
        });
        k_reduce_final<<<nv, kBT, 0, s>>>(part, nb, kNV, O2 + j0, 0);
    }
    // no synchronisation: out is ready in the order of `stream`
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}
