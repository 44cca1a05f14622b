// Two-level aggregation multigrid preconditioner with the Schwarz method as
// its smoother (arXiv:1502.04025, Sec. 2.4: the Krylov solver is
// preconditioned by a V-cycle whose smoother is the domain-decomposition
// preconditioner of Sec. 3).  The paper prints no formula for it; the reading:
//
//   aggregates  the Schwarz domains, each split by chirality (spins {0,1} and
//               {2,3}), so that the prolongator P commutes with gamma5
//   setup       nv caller-given random vectors w_k; setup_iters times each is
//               replaced by M_SAP w_k (setup_ncy cycles) and normalised; the
//               restriction of w_0..w_{nv-1} to every aggregate-chirality block
//               is orthonormalised (modified Gram-Schmidt, twice, FP64); the
//               block vectors are P's columns, stored in FP32
//   coarse      D_c = P^H D P: per aggregate a self block and one block per
//               hopping direction, (2 nv) x (2 nv) each, in FP32
//   V-cycle     e_c ~ D_c^{-1} P^H v by one GMRES cycle of coarse_iters steps
//               from zero, z = P e_c, r = v - D z, z += M_SAP(r) (post_ncy
//               cycles)
//   bootstrap   (the adaptive setup, `bootstrap` passes) each w_k becomes the
//               V-cycle of the method built so far applied to column k of P,
//               normalised; P and D_c are rebuilt from them
//
// The coarse problem is small (2 nv unknowns per domain), so its GMRES cycle
// runs without the host, captured once into a CUDA graph: per step one
// stencil launch (a CTA per domain) and one launch of an 8-CTA thread-block
// cluster that does the Gram-Schmidt dots, the update, the norm, the complex
// Givens rotation and the normalisation, its CTAs owning slices of the basis
// and exchanging partial sums through distributed shared memory; the
// least-squares solution is a back substitution at the end.
//
// Layouts: P as nv fine fields in the domain-blocked layout, so that the
// block (a, chi) of column k is the contiguous run of planes 6 chi .. 6 chi + 5
// of domain a; coarse vectors [domain slot][chi * nv + k]; the coarse
// operator [domain slot][9][2 nv columns][2 nv rows] (each block column-major,
// so that the threads of a stencil launch, one per row, read consecutive
// entries) with entry 0 the self block and entry 1 + dir the coupling to the
// neighbouring domain in direction dir.
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>

#include "dense.h"
#include "internal.h"

namespace qdd {

constexpr int kMgThreads = 256;

// bytes of one complex spinor entry in a storage precision
static size_t ebytes(qdd_prec p) { return p == QDD_PREC_F64 ? 16 : (p == QDD_PREC_F32 ? 8 : 4); }

// ------------------------------------------------------------ reductions

// Deterministic block sum of one double2 per thread: warp shuffles, then the
// warps' sums in order.  red holds kMgThreads/32 entries; every thread gets
// the total.
__device__ __forceinline__ double2 block_sum2(double2 v, double2 *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double2 t = make_double2(0, 0);
    for (int k = 0; k < nw; k++) {
        t.x += red[k].x;
        t.y += red[k].y;
    }
    return t;
}

// ------------------------------------------------------------ setup kernels

// Modified Gram-Schmidt, twice, over the nv vectors of one aggregate-chirality
// block (6 Vd contiguous complex entries of each vector), in FP64.
__global__ void __launch_bounds__(kMgThreads) k_mg_orth(double2 *w, int nv, int64_t stride, int Vd)
{
    __shared__ double2 red[kMgThreads / 32];
    const int d = blockIdx.x >> 1, chi = blockIdx.x & 1;
    const int64_t base = (int64_t)d * 12 * Vd + (int64_t)6 * chi * Vd;
    const int n = 6 * Vd;
    for (int pass = 0; pass < 2; pass++)
        for (int k = 0; k < nv; k++) {
            double2 *vk = w + k * stride + base;
            for (int l = 0; l < k; l++) {
                const double2 *vl = w + l * stride + base;
                double2 p = make_double2(0, 0);
                for (int e = threadIdx.x; e < n; e += blockDim.x) {
                    double2 a = vl[e], b = vk[e];
                    p.x += a.x * b.x + a.y * b.y;
                    p.y += a.x * b.y - a.y * b.x;
                }
                double2 c = block_sum2(p, red);  // <v_l, v_k>
                for (int e = threadIdx.x; e < n; e += blockDim.x) {
                    double2 a = vl[e], b = vk[e];
                    b.x -= c.x * a.x - c.y * a.y;
                    b.y -= c.x * a.y + c.y * a.x;
                    vk[e] = b;
                }
            }
            double2 p = make_double2(0, 0);
            for (int e = threadIdx.x; e < n; e += blockDim.x) p.x += vk[e].x * vk[e].x + vk[e].y * vk[e].y;
            double2 c = block_sum2(p, red);
            const double inv = c.x > 0 ? 1.0 / sqrt(c.x) : 0.0;
            for (int e = threadIdx.x; e < n; e += blockDim.x) vk[e] = make_double2(vk[e].x * inv, vk[e].y * inv);
        }
}

// Coarse operator, one CTA per aggregate (domain d), one thread per even/odd
// site pair.  For every coarse column j = (chi', k'): the basis vector b_j
// (column k' of P on chirality chi', on every aggregate) is hit by
//   self  A b_j(x) - kappa * (hops inside d)       (x in d, from b_j on d)
//   dir   -kappa * (the hop of x leaving d in dir)  (from b_j on the neighbour)
// and each part is projected on the columns i = (chi, k) of d:
//   Y[d][0][i][j] = <P_(d,i), self>,  Y[d][1 + dir][i][j] = <P_(d,i), dir part>.
// Per-warp partial sums go to shared memory and are added in warp order.
struct MgBasis {
    const float2 *P;
    int64_t stride;  // V * 12
    int Vd, nv;
    // b_j at (domain dd, site t): the chi' half of column k', the other half zero
    __device__ __forceinline__ void load(int j, int dd, int t, cpx<float> *x) const
    {
        const int chi = j / nv, k = j % nv;
        const float2 *p = P + k * stride + (int64_t)dd * 12 * Vd + t;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const bool on = (c / 6) == chi;
            float2 v = on ? __ldg(p + (int64_t)c * Vd) : make_float2(0.f, 0.f);
            x[c] = mk<float>(v.x, v.y);
        }
    }
};

template <int MU>
__device__ __forceinline__ void mg_hops_dir(const Geom &g, const Field<StF32> &U, const MgBasis &B, int j, int d,
                                            int s, const uint16_t *nb, bool crossing_only, int only_dir,
                                            cpx<float> *acc)
{
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const int dir = 2 * MU + b;
        const uint16_t e = nb[dir];
        const bool cross = (e & kCross) != 0;
        if (crossing_only ? (dir != only_dir || !cross) : cross) continue;
        const int nd = cross ? __ldg(g.nbd + d * 8 + dir) : d, ns = e & kSlotMask;
        if (!(QDD_IN_RANGE(nd, 0, g.Nd) && QDD_IN_RANGE(ns, 0, g.Vd))) continue;
        cpx<float> x[12], u[9];
        B.load(j, nd, ns, x);
        const float2 *up = U.p + ((int64_t)(b ? nd : d) * 36 + MU * 9) * g.Vd + (b ? ns : s);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float2 v = __ldg(up + (int64_t)k * g.Vd);
            u[k] = mk<float>(v.x, v.y);
        }
        if (b == 0) hop<MU, +1>(u, x, acc);
        else hop<MU, -1>(u, x, acc);
    }
}

__global__ void __launch_bounds__(kMgThreads) k_mg_coarse_build(Geom g, Field<StF32> U, Field<StF32> A, MgBasis B,
                                                                float kappa, float2 *Y)
{
    extern __shared__ float2 sRed[];  // [warps][9][2 nv]
    const int d = blockIdx.x, i = threadIdx.x, Vh = g.Vh, Vd = g.Vd;
    const int nc = 2 * B.nv, nw = blockDim.x >> 5, w = i >> 5;
    // the block is a whole number of warps; threads past the Vh site pairs
    // contribute zeros (their site indices are clamped to a valid one)
    const bool active = i < Vh;
    const int ii0 = active ? i : 0;
    const int sites[2] = {ii0, Vh + ii0};
    uint16_t nbs[2][8];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int k = 0; k < 8; k++) nbs[p][k] = __ldg(g.nbl + sites[p] * 8 + k);
    for (int j = 0; j < nc; j++) {
        for (int n = 0; n < 9; n++) {
            // part n of column j at this thread's two sites
            cpx<float> part[2][12];
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const int s = sites[p];
                cpx<float> acc[12];
#pragma unroll
                for (int k = 0; k < 12; k++) acc[k] = mk<float>(0, 0);
                const bool self = n == 0;
                const int od = n - 1;
                mg_hops_dir<0>(g, U, B, j, d, s, nbs[p], !self, od, acc);
                mg_hops_dir<1>(g, U, B, j, d, s, nbs[p], !self, od, acc);
                mg_hops_dir<2>(g, U, B, j, d, s, nbs[p], !self, od, acc);
                mg_hops_dir<3>(g, U, B, j, d, s, nbs[p], !self, od, acc);
#pragma unroll
                for (int k = 0; k < 12; k++) part[p][k] = (-kappa) * acc[k];
                if (self) {
                    cpx<float> x[12], y[12], m[18];
                    B.load(j, d, s, x);
                    const float2 *ap = A.p + (int64_t)d * 36 * Vd + s;
#pragma unroll
                    for (int blk = 0; blk < 2; blk++) {
#pragma unroll
                        for (int k = 0; k < 18; k++) {
                            float2 v = __ldg(ap + (int64_t)(blk * 18 + k) * Vd);
                            m[k] = mk<float>(v.x, v.y);
                        }
                        herm6_mul(m, x + 6 * blk, y + 6 * blk);
                    }
#pragma unroll
                    for (int k = 0; k < 12; k++) part[p][k] = part[p][k] + y[k];
                }
                if (!active) {
#pragma unroll
                    for (int k = 0; k < 12; k++) part[p][k] = mk<float>(0, 0);
                }
            }
            // projections on the columns of d
            for (int ii = 0; ii < nc; ii++) {
                const int chi = ii / B.nv, k = ii % B.nv;
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const float2 *pp = B.P + k * B.stride + (int64_t)d * 12 * Vd + (int64_t)6 * chi * Vd + sites[p];
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        float2 a = __ldg(pp + (int64_t)c * Vd);
                        cpx<float> b = part[p][6 * chi + c];
                        re = fmaf(a.x, b.re, fmaf(a.y, b.im, re));
                        im = fmaf(a.x, b.im, fmaf(-a.y, b.re, im));
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, o);
                    im += __shfl_xor_sync(0xffffffffu, im, o);
                }
                if ((i & 31) == 0) sRed[(w * 9 + n) * nc + ii] = make_float2(re, im);
            }
        }
        __syncthreads();
        for (int t = i; t < 9 * nc; t += blockDim.x) {
            double re = 0, im = 0;
            for (int ww = 0; ww < nw; ww++) {
                re += sRed[ww * 9 * nc + t].x;
                im += sRed[ww * 9 * nc + t].y;
            }
            const int n = t / nc, ii = t % nc;
            Y[(((int64_t)d * 9 + n) * nc + j) * nc + ii] = make_float2((float)re, (float)im);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ transfer

// rc[d][chi * nv + k] = <P_(d,chi,k), v>, one CTA per aggregate.  Each
// thread reads its entries of v once and accumulates all NV products (v is
// read once, P once); warp shuffles, then a fixed-order sum over the warps.
template <int NV, typename T2>
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict(const float2 *P, int64_t stride, int Vd, const T2 *v,
                                                            float2 *rc)
{
    __shared__ float2 part[kMgThreads / 32][NV];
    const int d = blockIdx.x, n = 6 * Vd;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int chi = 0; chi < 2; chi++) {
        const int64_t base = (int64_t)d * 12 * Vd + (int64_t)6 * chi * Vd;
        float px[NV], py[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) px[k] = py[k] = 0.f;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const T2 b = v[base + e];
            const float bx = (float)b.x, by = (float)b.y;
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const float2 a = __ldg(P + k * stride + base + e);
                px[k] = fmaf(a.x, bx, fmaf(a.y, by, px[k]));
                py[k] = fmaf(a.x, by, fmaf(-a.y, bx, py[k]));
            }
        }
#pragma unroll
        for (int k = 0; k < NV; k++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                px[k] += __shfl_xor_sync(0xffffffffu, px[k], o);
                py[k] += __shfl_xor_sync(0xffffffffu, py[k], o);
            }
            if (lane == 0) part[w][k] = make_float2(px[k], py[k]);
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            float2 t = part[0][threadIdx.x];
            for (int ww = 1; ww < nw; ww++) {
                t.x += part[ww][threadIdx.x].x;
                t.y += part[ww][threadIdx.x].y;
            }
            rc[(int64_t)d * 2 * NV + chi * NV + threadIdx.x] = t;
        }
        __syncthreads();  // part is rewritten for the other chirality
    }
}

template <typename T2>
static void launch_mg_restrict(int nv, int nd, const float2 *P, int64_t stride, int Vd, const T2 *v, float2 *rc,
                               cudaStream_t s)
{
    switch (nv) {
#define QDD_MG_RESTRICT(N) \
    case N: k_mg_restrict<N, T2><<<nd, kMgThreads, 0, s>>>(P, stride, Vd, v, rc); break;
        QDD_MG_RESTRICT(1) QDD_MG_RESTRICT(2) QDD_MG_RESTRICT(3) QDD_MG_RESTRICT(4)
        QDD_MG_RESTRICT(5) QDD_MG_RESTRICT(6) QDD_MG_RESTRICT(7) QDD_MG_RESTRICT(8)
        QDD_MG_RESTRICT(9) QDD_MG_RESTRICT(10) QDD_MG_RESTRICT(11) QDD_MG_RESTRICT(12)
        QDD_MG_RESTRICT(13) QDD_MG_RESTRICT(14) QDD_MG_RESTRICT(15) QDD_MG_RESTRICT(16)
#undef QDD_MG_RESTRICT
    default: break;  // nv is checked to be 1..16 at setup
    }
}

// z = P ec, one thread per fine complex entry
template <typename T2>
__global__ void k_mg_prolong(const float2 *P, int nv, int64_t stride, int Vd, const float2 *ec, T2 *z, int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int64_t d = e / (12 * Vd);
    const int chi = (int)((e - d * 12 * Vd) / Vd) / 6;
    const float2 *c = ec + d * 2 * nv + chi * nv;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nv; k++) {
        float2 a = __ldg(P + k * stride + e);
        float2 b = __ldg(c + k);
        re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
        im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
    }
    T2 out;
    out.x = re;
    out.y = im;
    z[e] = out;
}

// y = D_c x: y[d][i] = sum over the self block and the 8 neighbours of Y x.
// One CTA per domain; warp n applies block n (lanes over the rows, 2 nv <= 32),
// and the nine partial rows are added in block order in shared memory.
__global__ void __launch_bounds__(288) k_mg_coarse_apply(const float2 *Y, const int *nbd, int nc, const float2 *x,
                                                         float2 *y, const int *done)
{
    __shared__ float2 part[9][32];
    if (*done) return;  // the coarse cycle has broken down exactly: nothing left to do
    const int d = blockIdx.x, n = threadIdx.x >> 5, i = threadIdx.x & 31;
    float re = 0.f, im = 0.f;
    const int dn = (i < nc) ? (n == 0 ? d : __ldg(nbd + d * 8 + n - 1)) : d;
    if (i < nc && QDD_IN_RANGE(dn, 0, gridDim.x)) {
        const float2 *blk = Y + ((int64_t)d * 9 + n) * nc * nc + i;
        const float2 *xv = x + (int64_t)dn * nc;
#pragma unroll 8
        for (int j = 0; j < nc; j++) {
            float2 a = __ldg(blk + (int64_t)j * nc), b = xv[j];
            re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
            im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
        }
    }
    part[n][i] = make_float2(re, im);
    __syncthreads();
    if (threadIdx.x < nc) {
        float2 t = part[0][threadIdx.x];
        for (int k = 1; k < 9; k++) {
            t.x += part[k][threadIdx.x].x;
            t.y += part[k][threadIdx.x].y;
        }
        y[(int64_t)d * nc + threadIdx.x] = t;
    }
}

// ------------------------------------------------------------ coarse GMRES

constexpr int kCgThreads = 1024;
constexpr int kCgMaxM = 64;

// State of one coarse GMRES cycle: Givens rotations, the rotated right-hand
// side g and the triangular R (column-major, kCgMaxM x kCgMaxM).  FP32, like
// the rest of the coarse cycle: the single thread that updates it would pay
// the FP64 pipe's latency on every step.
struct CgState {
    float cs[kCgMaxM];
    float2 sn[kCgMaxM];
    float2 g[kCgMaxM + 1];
    float2 R[kCgMaxM * kCgMaxM];
    int jm;    // columns in use
    int done;  // an exact breakdown ended the cycle
};

__device__ __forceinline__ float2 block_sum_f2(float2 v, float2 *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
        t.x += red[k].x;
        t.y += red[k].y;
    }
    return t;
}

// v_0 = b / |b|, g = (|b|, 0, ...)
__global__ void __launch_bounds__(kCgThreads) k_mg_cg_init(const float2 *b, float2 *V, int64_t n, CgState *st)
{
    __shared__ float2 red[kCgThreads / 32];
    float2 p = make_float2(0.f, 0.f);
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) p.x += b[e].x * b[e].x + b[e].y * b[e].y;
    const float beta = sqrtf(block_sum_f2(p, red).x);
    const float inv = beta > 0.f ? 1.f / beta : 0.f;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) V[e] = make_float2(b[e].x * inv, b[e].y * inv);
    if (threadIdx.x == 0) {
        for (int k = 0; k <= kCgMaxM; k++) st->g[k] = make_float2(0.f, 0.f);
        st->g[0] = make_float2(beta, 0.f);
        st->jm = 0;
        st->done = beta > 0.f ? 0 : 1;
    }
}

// Step j: w = V_{j+1} (already D_c V_j) is orthogonalised against V_0..V_j
// (classical Gram-Schmidt), h_{j+1,j} = |w|, V_{j+1} = w / |w|, and column j
// of the Hessenberg matrix is rotated into R (complex Givens rotations
// G = [[c, s], [-conj(s), c]], c real).
//
// One thread-block cluster of kCgCluster CTAs (one per SM): each CTA owns a
// slice of the vectors; partial dot products and norms are exchanged through
// distributed shared memory between cluster barriers, and every CTA adds the
// partials in rank order, so all of them hold the same h.
constexpr int kCgCluster = 8;
constexpr int kCgClThreads = 512;

__global__ void __cluster_dims__(kCgCluster, 1, 1) __launch_bounds__(kCgClThreads)
    k_mg_cg_step(float2 *V, int j, int64_t n, CgState *st)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ float2 sdot[kCgMaxM][kCgClThreads / 32];
    __shared__ float2 hpart[kCgMaxM + 1];  // this CTA's partial dots, then [kCgMaxM] its partial |w|^2
    __shared__ float2 h[kCgMaxM];
    __shared__ float2 red[kCgClThreads / 32];
    __shared__ float s_cs[kCgMaxM];
    __shared__ float2 s_sn[kCgMaxM], s_col[kCgMaxM + 1];
    if (st->done) return;  // uniform over the cluster: every CTA leaves before any barrier
    const int rank = (int)cl.block_rank();
    const int64_t chunk = (n + kCgCluster - 1) / kCgCluster;
    const int64_t lo = rank * chunk, hi = lo + chunk < n ? lo + chunk : n;
    float2 *w = V + (int64_t)(j + 1) * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // partial dot products over this CTA's slice, 16 at a time
    for (int i0 = 0; i0 <= j; i0 += 16) {
        float2 acc[16];
#pragma unroll
        for (int q = 0; q < 16; q++) acc[q] = make_float2(0.f, 0.f);
        for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            const float2 b = w[e];
#pragma unroll
            for (int q = 0; q < 16; q++)
                if (i0 + q <= j) {
                    const float2 a = V[(int64_t)(i0 + q) * n + e];
                    acc[q].x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[q].x));
                    acc[q].y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc[q].y));
                }
        }
#pragma unroll
        for (int q = 0; q < 16; q++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
            }
            if (lane == 0 && i0 + q <= j) sdot[i0 + q][wid] = acc[q];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        float2 t = make_float2(0.f, 0.f);
        for (int k = 0; k < nwarp; k++) {
            t.x += sdot[i][k].x;
            t.y += sdot[i][k].y;
        }
        hpart[i] = t;
    }
    // the rotations so far, for the Givens step on rank 0
    if (rank == 0)
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            s_cs[i] = st->cs[i];
            s_sn[i] = st->sn[i];
        }
    cl.sync();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        float2 t = make_float2(0.f, 0.f);
        for (int r = 0; r < kCgCluster; r++) {
            const float2 v = cl.map_shared_rank(hpart, r)[i];
            t.x += v.x;
            t.y += v.y;
        }
        h[i] = t;
    }
    __syncthreads();
    // w -= sum h_i V_i on this slice, and its partial norm
    float2 p = make_float2(0.f, 0.f);
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        float2 x = w[e];
        for (int i = 0; i <= j; i++) {
            const float2 a = V[(int64_t)i * n + e], c = h[i];
            x.x -= c.x * a.x - c.y * a.y;
            x.y -= c.x * a.y + c.y * a.x;
        }
        w[e] = x;
        p.x += x.x * x.x + x.y * x.y;
    }
    p = block_sum_f2(p, red);
    if (threadIdx.x == 0) hpart[kCgMaxM] = p;  // its own slot: the dot partials stay readable
    cl.sync();
    float hn2 = 0.f;
    for (int r = 0; r < kCgCluster; r++) hn2 += cl.map_shared_rank(hpart, r)[kCgMaxM].x;
    const float hn = sqrtf(hn2);
    const float inv = hn > 0.f ? 1.f / hn : 0.f;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) w[e] = make_float2(w[e].x * inv, w[e].y * inv);
    if (rank == 0 && threadIdx.x == 0) {
        const float2 gj = st->g[j];
        float2 *col = s_col;
        for (int i = 0; i <= j; i++) col[i] = h[i];
        col[j + 1] = make_float2(hn, 0.f);
        for (int i = 0; i < j; i++) {
            const float c = s_cs[i];
            const float2 sv = s_sn[i], a = col[i], b = col[i + 1];
            // (a, b) <- (c a + s b, -conj(s) a + c b)
            col[i] = make_float2(c * a.x + sv.x * b.x - sv.y * b.y, c * a.y + sv.x * b.y + sv.y * b.x);
            col[i + 1] = make_float2(c * b.x - (sv.x * a.x + sv.y * a.y), c * b.y - (sv.x * a.y - sv.y * a.x));
        }
        const float2 a = col[j];
        const float bb = hn;  // real, >= 0
        const float aa = sqrtf(a.x * a.x + a.y * a.y);
        const float r = sqrtf(aa * aa + bb * bb);
        float c;
        float2 sv;
        if (aa == 0.f) {
            c = 0.f;
            sv = make_float2(1.f, 0.f);
        } else {
            c = aa / r;
            sv = make_float2(a.x / aa * bb / r, a.y / aa * bb / r);
        }
        st->cs[j] = c;
        st->sn[j] = sv;
        col[j] = aa == 0.f ? make_float2(bb, 0.f) : make_float2(a.x / aa * r, a.y / aa * r);
        st->g[j] = make_float2(c * gj.x, c * gj.y);
        st->g[j + 1] = make_float2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
        st->jm = j + 1;
        if (!(hn > 0.f)) st->done = 1;
    }
    if (rank == 0) {
        __syncthreads();
        for (int i = threadIdx.x; i <= j; i += blockDim.x) st->R[j * kCgMaxM + i] = s_col[i];
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// x = V y with R y = g (back substitution), over the st->jm columns in use;
// every CTA solves the small triangular system from a shared-memory copy and
// combines its slice of the vectors
__global__ void __launch_bounds__(256) k_mg_cg_finish(const float2 *V, int64_t n, const CgState *st, float2 *x, int m)
{
    extern __shared__ float2 sR[];  // [m][m]: column k at k * m (jm <= m)
    __shared__ float2 y[kCgMaxM];
    __shared__ float2 sg[kCgMaxM];
    const int jm = st->jm;
    for (int t = threadIdx.x; t < jm * m; t += blockDim.x) {
        const int k = t / m, i = t % m;
        sR[t] = i <= k ? st->R[k * kCgMaxM + i] : make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < jm; t += blockDim.x) sg[t] = st->g[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = jm - 1; i >= 0; i--) {
            float2 t = sg[i];
            for (int k = i + 1; k < jm; k++) {
                const float2 r = sR[k * m + i], yk = y[k];
                t.x -= r.x * yk.x - r.y * yk.y;
                t.y -= r.x * yk.y + r.y * yk.x;
            }
            const float2 d = sR[i * m + i];
            const float dn = d.x * d.x + d.y * d.y;
            y[i] = dn > 0.f ? make_float2((t.x * d.x + t.y * d.y) / dn, (t.y * d.x - t.x * d.y) / dn)
                            : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int k = 0; k < jm; k++) {
            float2 a = V[(int64_t)k * n + e], c = y[k];
            re = fmaf(c.x, a.x, fmaf(-c.y, a.y, re));
            im = fmaf(c.x, a.y, fmaf(c.y, a.x, im));
        }
        x[e] = make_float2(re, im);
    }
}

// out = a - b
__global__ void k_mg_sub(const double2 *a, const double2 *b, double2 *out, int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

// ------------------------------------------------------------ host side

struct Multigrid {
    qdd_mg_params p{};
    int nv = 0, nc = 0;  // coarse dof per aggregate, nc = 2 nv
    int64_t ncoarse = 0; // Nd * nc
    DevMem P;            // nv fine fields, FP32, domain layout
    DevMem Y;            // coarse operator
    // V-cycle work: FP64 fine temporaries, Schwarz residual and face slots,
    // coarse GMRES basis and scalars
    DevMem t64, r64, rho, rho_s, face, err;
    DevMem cV, cx, cb, cst;  // coarse GMRES basis (coarse_iters + 1 vectors), solution, rhs, CgState
    DevMem api_v, api_z, api_io;  // qdd_mg_vcycle's input, output and host-transfer buffers (kept, so
                                  // that a call allocates and frees nothing after the first)
    cudaStream_t cap = nullptr;       // stream the coarse cycle was captured on
    cudaGraph_t graph = nullptr;      // the coarse cycle: init, coarse_iters x (stencil, step), finish
    cudaGraphExec_t exec = nullptr;
    ~Multigrid()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

static qdd_status mg_sap(Gauge *g, Multigrid &M, qdd_prec sp, const double2 *src64, void *psi, bool accumulate,
                         int ncy, cudaStream_t s)
{
    // rho = src in the smoother's storage, psi (+)= M_SAP rho
    QDD_TRY(launch_spinor_convert(g, src64, nullptr, QDD_PREC_F64, M.rho.p, M.rho_s.as<float>(), spinor_store(sp), 1,
                                  s));
    SapBuffers sb{M.rho.p, M.face.p, psi, M.rho_s.as<float>()};
    SeqScope seq(g->ctx->timer, K_SAP, s);
    for (int hs = 0; hs < 2 * ncy; hs++)
        QDD_TRY(launch_sap_halfsweep(g, sp, sb, hs & 1, M.p.nmr, 1, accumulate ? 0 : (hs < 2), hs >= 1, 0,
                                     M.err.as<int>(), s, hs >= 1, false));
    return QDD_OK;
}

// The launches of one coarse GMRES cycle (cx ~ D_c^{-1} cb, coarse_iters
// steps from zero), recorded once into a CUDA graph.
static void mg_coarse_launches(Gauge *g, Multigrid &M, cudaStream_t s)
{
    const int64_t n = M.ncoarse;
    const int m = M.p.coarse_iters;
    float2 *V = M.cV.as<float2>();
    CgState *st = M.cst.as<CgState>();
    k_mg_cg_init<<<1, kCgThreads, 0, s>>>(M.cb.as<float2>(), V, n, st);
    for (int j = 0; j < m; j++) {
        k_mg_coarse_apply<<<g->hg.Nd, 288, 0, s>>>(M.Y.as<float2>(), g->geom.nbd, M.nc, V + (int64_t)j * n,
                                                   V + (int64_t)(j + 1) * n, &st->done);
        k_mg_cg_step<<<kCgCluster, kCgClThreads, 0, s>>>(V, j, n, st);
    }
    k_mg_cg_finish<<<(int)std::min<int64_t>((n + 255) / 256, 304), 256, (size_t)m * m * sizeof(float2), s>>>(
        V, n, st, M.cx.as<float2>(), m);
}

static qdd_status mg_capture(Gauge *g, Multigrid &M)
{
    const int m = M.p.coarse_iters;
    QDD_CUDA(cudaFuncSetAttribute(k_mg_cg_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((size_t)m * m * sizeof(float2))));
    QDD_CUDA(cudaStreamCreateWithFlags(&M.cap, cudaStreamNonBlocking));
    QDD_CUDA(cudaStreamBeginCapture(M.cap, cudaStreamCaptureModeThreadLocal));
    mg_coarse_launches(g, M, M.cap);
    QDD_CUDA(cudaStreamEndCapture(M.cap, &M.graph));
    QDD_CUDA(cudaGraphInstantiate(&M.exec, M.graph, 0));
    return QDD_OK;
}

// cx ~ D_c^{-1} cb: replay the captured coarse cycle on the caller's stream
static qdd_status mg_coarse_solve(Gauge *g, Multigrid &M, cudaStream_t s)
{
    LaunchScope ls(g->ctx->timer, K_SAP, s, false);
    QDD_CUDA(cudaGraphLaunch(M.exec, s));
    for (int k = 1; k < 2 * M.p.coarse_iters + 2; k++) g->ctx->timer.count(K_SAP);  // the scope counted one
    return QDD_OK;
}

// z = M_MG v for one right-hand side: v FP64 (domain layout, not M's own
// buffers), z in zp storage.
static qdd_status mg_vcycle_with(Gauge *g, Multigrid &M, const double2 *v, void *z, qdd_prec zp, cudaStream_t s)
{
    const int64_t nfine = (int64_t)g->hg.V * 12;
    const int64_t stride = nfine;
    {
        LaunchScope ls(g->ctx->timer, K_SAP, s);
        launch_mg_restrict<double2>(M.nv, g->hg.Nd, M.P.as<float2>(), stride, g->hg.Vd, v, M.cb.as<float2>(), s);
        QDD_CUDA(cudaGetLastError());
    }
    QDD_TRY(mg_coarse_solve(g, M, s));
    {
        LaunchScope ls(g->ctx->timer, K_SAP, s);
        const int nb = (int)((nfine + 255) / 256);
        if (zp == QDD_PREC_F64)
            k_mg_prolong<double2><<<nb, 256, 0, s>>>(M.P.as<float2>(), M.nv, stride, g->hg.Vd, M.cx.as<float2>(),
                                                     (double2 *)z, nfine);
        else
            k_mg_prolong<float2><<<nb, 256, 0, s>>>(M.P.as<float2>(), M.nv, stride, g->hg.Vd, M.cx.as<float2>(),
                                                    (float2 *)z, nfine);
        QDD_CUDA(cudaGetLastError());
    }
    if (M.p.post_ncy > 0) {
        // r = v - D z, then z += M_SAP r
        const qdd_prec ar = zp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
        QDD_TRY(launch_dslash(g, ar, ar, z, nullptr, zp, M.t64.p, nullptr, QDD_PREC_F64, nullptr, 1, s));
        {
            LaunchScope ls(g->ctx->timer, K_SAP, s);
            k_mg_sub<<<(int)((nfine + 255) / 256), 256, 0, s>>>(v, M.t64.as<double2>(), M.r64.as<double2>(), nfine);
            QDD_CUDA(cudaGetLastError());
        }
        QDD_TRY(mg_sap(g, M, M.p.sap_prec, M.r64.as<double2>(), z, true, M.p.post_ncy, s));
    }
    return QDD_OK;
}

qdd_status mg_vcycle(Gauge *g, const double2 *v, void *z, qdd_prec zp, cudaStream_t s)
{
    return mg_vcycle_with(g, *g->mg, v, z, zp, s);
}

// The prolongator and coarse operator from test vectors w64 (nv FP64 fields,
// overwritten): per aggregate and chirality the vectors are orthonormalised,
// P takes them in FP32, and D_c = P^H D P is rebuilt.  The captured coarse
// cycle reads D_c in place, so it stays valid.
static qdd_status mg_build(Gauge *g, Multigrid &M, double2 *w64, cudaStream_t s)
{
    const HostGeom &hg = g->hg;
    const int64_t nfine = (int64_t)hg.V * 12;
    k_mg_orth<<<hg.Nd * 2, kMgThreads, 0, s>>>(w64, M.nv, nfine, hg.Vd);
    QDD_CUDA(cudaGetLastError());
    QDD_TRY(launch_spinor_convert(g, w64, nullptr, QDD_PREC_F64, M.P.p, nullptr, QDD_PREC_F32, M.nv, s));
    PrecCopy &c = g->copies[QDD_PREC_F32];
    MgBasis B{M.P.as<float2>(), nfine, hg.Vd, M.nv};
    const int bthreads = (hg.Vh + 31) / 32 * 32;
    const size_t smem = (size_t)(bthreads / 32) * 9 * M.nc * sizeof(float2);
    QDD_CUDA(cudaFuncSetAttribute(k_mg_coarse_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mg_coarse_build<<<hg.Nd, bthreads, smem, s>>>(g->geom, Field<StF32>{c.links.as<float2>(), nullptr},
                                                  Field<StF32>{c.clov.as<float2>(), nullptr}, B, (float)g->kappa,
                                                  M.Y.as<float2>());
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_prec mg_smoother_prec(const Gauge *g) { return g->mg ? g->mg->p.sap_prec : QDD_PREC_F32; }

// out-of-range indices the kernels of this file have skipped (QDD_CHECK builds)
unsigned long long check_hits_mg()
{
#ifdef QDD_CHECK
    unsigned long long h = 0;
    if (cudaMemcpyFromSymbol(&h, g_check_hits, sizeof(h)) != cudaSuccess) return ~0ull;
    return h;
#else
    return 0;
#endif
}

static qdd_status mg_check(const qdd_mg_params *p)
{
    if (!p || p->nv < 1 || p->nv > 16 || p->setup_iters < 0 || p->setup_ncy < 1 || p->nmr < 0 || p->post_ncy < 0 ||
        p->coarse_iters < 1 || p->coarse_iters > kCgMaxM || !is_sap_prec(p->sap_prec) || p->bootstrap < 0 ||
        p->bootstrap > 8) {
        set_error("invalid multigrid parameters");
        return QDD_EINVAL;
    }
    return QDD_OK;
}

}  // namespace qdd

using namespace qdd;

extern "C" {

void qdd_mg_default_params(qdd_mg_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nv = 8;
    p->setup_iters = 3;
    p->setup_ncy = 2;
    p->nmr = 4;
    p->post_ncy = 2;
    p->coarse_iters = 12;
    p->sap_prec = QDD_PREC_F32;
}

qdd_status qdd_mg_setup(qdd_gauge *g, const qdd_mg_params *p, const double *w0, int on_device)
{
    clear_error();
    if (!g || !w0) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    QDD_TRY(mg_check(p));
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    if (g->slab) {
        set_error("the multigrid preconditioner is built on unsharded gauge fields only");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    Ctx *ctx = g->ctx;
    QDD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = nullptr;
    const HostGeom &hg = g->hg;
    const int nv = p->nv;
    const int64_t nfine = (int64_t)hg.V * 12;
    auto M = std::make_shared<Multigrid>();
    M->p = *p;
    M->nv = nv;
    M->nc = 2 * nv;
    M->ncoarse = (int64_t)hg.Nd * M->nc;
    const qdd_prec sp = p->sap_prec;
    const qdd_prec zp = sp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    QDD_TRY(M->P.alloc(ctx, (size_t)nv * nfine * sizeof(float2)));
    QDD_TRY(M->Y.alloc(ctx, (size_t)hg.Nd * 9 * M->nc * M->nc * sizeof(float2)));
    QDD_TRY(M->t64.alloc(ctx, nfine * sizeof(double2)));
    QDD_TRY(M->r64.alloc(ctx, nfine * sizeof(double2)));
    QDD_TRY(M->rho.alloc(ctx, nfine * ebytes(spinor_store(sp))));
    if (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S) QDD_TRY(M->rho_s.alloc(ctx, hg.V * sizeof(float)));
    QDD_TRY(M->face.alloc(ctx, sap_face_bytes(hg, sp, 1)));
    QDD_TRY(M->err.alloc(ctx, sizeof(int)));
    QDD_CUDA(cudaMemset(M->err.p, 0, sizeof(int)));
    QDD_TRY(M->cV.alloc(ctx, (size_t)(p->coarse_iters + 1) * M->ncoarse * sizeof(float2)));
    QDD_TRY(M->cx.alloc(ctx, M->ncoarse * sizeof(float2)));
    QDD_TRY(M->cb.alloc(ctx, M->ncoarse * sizeof(float2)));
    QDD_TRY(M->cst.alloc(ctx, sizeof(CgState)));
    DevMem dscr, ddev;  // setup normalisation
    QDD_TRY(blas_scratch_ensure(ctx, dscr));
    QDD_TRY(ddev.alloc(ctx, sizeof(double2)));
    QDD_TRY(ensure_copy(g, QDD_PREC_F32, s));
    if (zp == QDD_PREC_F32 || sp != QDD_PREC_F64) QDD_TRY(ensure_copy(g, sp, s));

    // the test vectors in FP64, domain layout
    DevMem w64, io, zt;
    QDD_TRY(w64.alloc(ctx, (size_t)nv * nfine * sizeof(double2)));
    QDD_TRY(zt.alloc(ctx, nfine * ebytes(zp)));
    const double *src = w0;
    if (!on_device) {
        QDD_TRY(io.alloc(ctx, (size_t)nv * nfine * sizeof(double2)));
        QDD_CUDA(cudaMemcpy(io.p, w0, (size_t)nv * nfine * sizeof(double2), cudaMemcpyHostToDevice));
        src = io.as<double>();
    }
    QDD_TRY(launch_spinor_in(g, src, w64.p, nullptr, QDD_PREC_F64, nv, s));
    io.release();
    g->mg.reset();  // an earlier preconditioner is replaced; this one is published when complete
    double2 *dev = ddev.as<double2>(), *scr = dscr.as<double2>();
    for (int it = 0; it < p->setup_iters; it++)
        for (int k = 0; k < nv; k++) {
            double2 *wk = w64.as<double2>() + k * nfine;
            QDD_TRY(mg_sap(g, *M, sp, wk, zt.p, false, p->setup_ncy, s));
            QDD_TRY(launch_spinor_convert(g, zt.p, nullptr, zp, wk, nullptr, QDD_PREC_F64, 1, s));
            QDD_TRY(blas_norm2(ctx, wk, nfine, dev, scr, s));
            QDD_TRY(blas_scale_by_norm(ctx, wk, nfine, dev, wk, s));
        }
    QDD_TRY(mg_build(g, *M, w64.as<double2>(), s));
    QDD_TRY(mg_capture(g, *M));
    // bootstrap (the adaptive setup): each test vector becomes the V-cycle of
    // the two-level method just built applied to its prolongator column,
    // normalised; P and D_c are rebuilt from them
    if (p->bootstrap > 0) {
        DevMem vin;
        QDD_TRY(vin.alloc(ctx, nfine * sizeof(double2)));
        for (int b = 0; b < p->bootstrap; b++) {
            for (int k = 0; k < nv; k++) {
                double2 *wk = w64.as<double2>() + k * nfine;
                QDD_TRY(launch_spinor_convert(g, M->P.as<float2>() + k * nfine, nullptr, QDD_PREC_F32, vin.p,
                                              nullptr, QDD_PREC_F64, 1, s));
                QDD_TRY(mg_vcycle_with(g, *M, vin.as<double2>(), zt.p, zp, s));
                QDD_TRY(launch_spinor_convert(g, zt.p, nullptr, zp, wk, nullptr, QDD_PREC_F64, 1, s));
                QDD_TRY(blas_norm2(ctx, wk, nfine, dev, scr, s));
                QDD_TRY(blas_scale_by_norm(ctx, wk, nfine, dev, wk, s));
            }
            QDD_TRY(mg_build(g, *M, w64.as<double2>(), s));
        }
    }
    QDD_CUDA(cudaStreamSynchronize(s));
    int herr = 0;
    QDD_CUDA(cudaMemcpy(&herr, M->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        set_error("Schwarz smoother error flag %d during the multigrid setup", herr);
        return QDD_ECUDA;
    }
    g->mg = M;
    return QDD_OK;
}

qdd_status qdd_mg_vcycle(qdd_gauge *g, const double *v, double *z, int on_device, void *stream)
{
    clear_error();
    if (!g || !v || !z) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    if (!g->mg) {
        set_error("qdd_mg_setup has not been called");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    Ctx *ctx = g->ctx;
    QDD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nfine = (int64_t)g->hg.V * 12;
    const qdd_prec zp = g->mg->p.sap_prec == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    Multigrid &M = *g->mg;
    DevMem &io = M.api_io, &vin = M.api_v, &zt = M.api_z;
    QDD_TRY(vin.ensure(ctx, nfine * sizeof(double2)));
    QDD_TRY(zt.ensure(ctx, nfine * ebytes(zp)));
    const double *src = v;
    if (!on_device) {
        QDD_TRY(io.ensure(ctx, nfine * sizeof(double2)));
        QDD_CUDA(cudaMemcpyAsync(io.p, v, nfine * sizeof(double2), cudaMemcpyHostToDevice, s));
        src = io.as<double>();
    }
    QDD_TRY(launch_spinor_in(g, src, vin.p, nullptr, QDD_PREC_F64, 1, s));
    QDD_TRY(mg_vcycle(g, vin.as<double2>(), zt.p, zp, s));
    double *dst = z;
    if (!on_device) {
        QDD_TRY(io.ensure(ctx, nfine * sizeof(double2)));
        dst = io.as<double>();
    }
    QDD_TRY(launch_spinor_out(g, zt.p, nullptr, dst, zp, 1, s));
    if (!on_device) QDD_CUDA(cudaMemcpyAsync(z, dst, nfine * sizeof(double2), cudaMemcpyDeviceToHost, s));
    QDD_CUDA(cudaStreamSynchronize(s));
    return QDD_OK;
}

qdd_status qdd_mg_get_basis(qdd_gauge *g, double *out)
{
    clear_error();
    if (!g || !out) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    if (!g->mg) {
        set_error("qdd_mg_setup has not been called");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    Ctx *ctx = g->ctx;
    QDD_CUDA(cudaSetDevice(ctx->device));
    const int64_t nfine = (int64_t)g->hg.V * 12;
    const int nv = g->mg->nv;
    DevMem io;
    QDD_TRY(io.alloc(ctx, (size_t)nv * nfine * sizeof(double2)));
    QDD_TRY(launch_spinor_out(g, g->mg->P.p, nullptr, io.as<double>(), QDD_PREC_F32, nv, nullptr));
    QDD_CUDA(cudaMemcpy(out, io.p, (size_t)nv * nfine * sizeof(double2), cudaMemcpyDeviceToHost));
    return QDD_OK;
}

}  // extern "C"
