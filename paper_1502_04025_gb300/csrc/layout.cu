// Domain decomposition geometry and field layout conversions.
//
// The lattice is split into domains of dom[0..3] sites (arXiv:1502.04025,
// Sec. 3.1 and Sec. 3.3: 4^4 and 8x4^3 domains), coloured like a
// checkerboard so that the domains of one colour are independent (Sec. 3.5,
// footnote: n_d = N_d/2 domains can be processed at once).  Each domain's
// data is one contiguous, plane-major block in device memory (Sec. 3.2
// motivates choosing the layout for the algorithm; here it serves coalesced
// warps and single bulk copies into shared memory).
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace qdd {

// ----------------------------------------------------------------- geometry

static void local_coords(const int dom[4], int Vh, int s, int c[4])
{
    int p = s >= Vh;
    int h = s - p * Vh;
    int l = 2 * h;
    c[0] = l % dom[0];
    l /= dom[0];
    c[1] = l % dom[1];
    l /= dom[1];
    c[2] = l % dom[2];
    c[3] = l / dom[2];
    c[0] += (p + c[1] + c[2] + c[3]) & 1;
}

static int local_slot(const int dom[4], int Vh, const int c[4])
{
    int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    int l = c[0] + dom[0] * (c[1] + dom[1] * (c[2] + dom[2] * c[3]));
    return p * Vh + (l >> 1);
}

qdd_status make_geometry(const int L[4], const int dom[4], HostGeom &hg)
{
    long long V = 1;
    hg.Vd = 1;
    hg.Nd = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (L[mu] <= 0 || dom[mu] < 2 || dom[mu] % 2 || L[mu] % dom[mu]) {
            set_error("invalid geometry: L[%d]=%d dom[%d]=%d (dom must be even and divide L)", mu, L[mu], mu,
                      dom[mu]);
            return QDD_EINVAL;
        }
        int nb = L[mu] / dom[mu];
        if (nb < 2 || nb % 2) {
            set_error("invalid geometry: L[%d]/dom[%d] = %d blocks; need an even number >= 2", mu, mu, nb);
            return QDD_EINVAL;
        }
        hg.L[mu] = L[mu];
        hg.dom[mu] = dom[mu];
        hg.nb[mu] = nb;
        V *= L[mu];
        hg.Vd *= dom[mu];
        hg.Nd *= nb;
    }
    if (hg.Vd > 512) {
        set_error("domain volume %d exceeds 512 sites", hg.Vd);
        return QDD_EINVAL;
    }
    if (V > (1LL << 30)) {
        set_error("lattice volume %lld too large", V);
        return QDD_EINVAL;
    }
    hg.V = (int)V;
    hg.Vh = hg.Vd / 2;
    hg.Nd2 = hg.Nd / 2;

    // slot <-> block: slot = colour*Nd/2 + (block >> 1)
    hg.slot_block.assign(hg.Nd, -1);
    hg.block_slot.assign(hg.Nd, -1);
    std::vector<int> &block_slot = hg.block_slot;
    for (int b = 0; b < hg.Nd; b++) {
        int bc[4], t = b;
        for (int mu = 0; mu < 4; mu++) {
            bc[mu] = t % hg.nb[mu];
            t /= hg.nb[mu];
        }
        int colour = (bc[0] + bc[1] + bc[2] + bc[3]) & 1;
        int slot = colour * hg.Nd2 + (b >> 1);
        hg.slot_block[slot] = b;
        block_slot[b] = slot;
    }
    for (int d = 0; d < hg.Nd; d++)
        if (hg.slot_block[d] < 0) {
            set_error("internal error: domain slot map is not a bijection");
            return QDD_EINVAL;
        }

    // local neighbour table
    hg.nbl.assign((size_t)hg.Vd * 8, 0);
    for (int s = 0; s < hg.Vd; s++) {
        int c[4];
        local_coords(hg.dom, hg.Vh, s, c);
        if (local_slot(hg.dom, hg.Vh, c) != s) {
            set_error("internal error: site slot map is not a bijection");
            return QDD_EINVAL;
        }
        for (int mu = 0; mu < 4; mu++)
            for (int b = 0; b < 2; b++) {
                int cc[4] = {c[0], c[1], c[2], c[3]};
                cc[mu] += b ? -1 : 1;
                uint16_t cross = 0;
                if (cc[mu] < 0 || cc[mu] >= hg.dom[mu]) {
                    cc[mu] = (cc[mu] + hg.dom[mu]) % hg.dom[mu];
                    cross = kCross;
                }
                hg.nbl[(size_t)s * 8 + 2 * mu + b] = (uint16_t)(local_slot(hg.dom, hg.Vh, cc) | cross);
            }
    }
    // face slots: the hops that leave a domain, direction by direction; within
    // direction mu (either sign) a site's slot is the lexicographic index of
    // its coordinates transverse to mu, shared by the site across the face
    hg.nf = 0;
    for (int dir = 0; dir < 8; dir++) {
        hg.foff[dir] = hg.nf;
        hg.nf += hg.Vd / hg.dom[dir >> 1];
    }
    hg.fcoord.assign(hg.Vd, 0);
    for (int s = 0; s < hg.Vd; s++) {
        int c[4];
        local_coords(hg.dom, hg.Vh, s, c);
        uint32_t packed = 0;
        for (int mu = 0; mu < 4; mu++) {
            int t = 0, stride = 1;
            for (int nu = 0; nu < 4; nu++)
                if (nu != mu) {
                    t += c[nu] * stride;
                    stride *= hg.dom[nu];
                }
            packed |= (uint32_t)t << (8 * mu);  // t < Vd / dom[mu] <= 256
        }
        hg.fcoord[s] = packed;
    }
    // domain neighbour table
    hg.nbd.assign((size_t)hg.Nd * 8, 0);
    for (int d = 0; d < hg.Nd; d++) {
        int b = hg.slot_block[d], bc[4], t = b;
        for (int mu = 0; mu < 4; mu++) {
            bc[mu] = t % hg.nb[mu];
            t /= hg.nb[mu];
        }
        for (int mu = 0; mu < 4; mu++)
            for (int st = 0; st < 2; st++) {
                int cc[4] = {bc[0], bc[1], bc[2], bc[3]};
                cc[mu] = (cc[mu] + (st ? -1 : 1) + hg.nb[mu]) % hg.nb[mu];
                int nbk = cc[0] + hg.nb[0] * (cc[1] + hg.nb[1] * (cc[2] + hg.nb[2] * cc[3]));
                hg.nbd[(size_t)d * 8 + 2 * mu + st] = block_slot[nbk];
            }
    }
    // internal index -> host site index
    hg.site_of.assign(hg.V, 0);
    for (int d = 0; d < hg.Nd; d++) {
        int b = hg.slot_block[d], bc[4], t = b;
        for (int mu = 0; mu < 4; mu++) {
            bc[mu] = t % hg.nb[mu];
            t /= hg.nb[mu];
        }
        for (int s = 0; s < hg.Vd; s++) {
            int c[4];
            local_coords(hg.dom, hg.Vh, s, c);
            int x[4];
            for (int mu = 0; mu < 4; mu++) x[mu] = bc[mu] * hg.dom[mu] + c[mu];
            hg.site_of[(size_t)d * hg.Vd + s] = x[0] + hg.L[0] * (x[1] + hg.L[1] * (x[2] + hg.L[2] * x[3]));
        }
    }
    return QDD_OK;
}

// ------------------------------------------------------------------ kernels

template <typename S>
__device__ __forceinline__ void store_spinor(Field<S> f, int64_t base, int64_t sbase, int Vd, int d, int s,
                                             const cpx<double> *v)
{
    typename S::T2 *p = f.p + base + (int64_t)d * 12 * Vd + s;
    if (S::kScaled) {
        double m = 0;
        for (int k = 0; k < 12; k++) m = fmax(m, fmax(fabs(v[k].re), fabs(v[k].im)));
        float sc = (float)m;
        double inv = m > 0 ? 1.0 / (double)sc : 0.0;
        f.scale[sbase + (int64_t)d * Vd + s] = sc;
        if constexpr (S::kQuad) {
            cpx<double> y[12];
            for (int k = 0; k < 12; k++) y[k] = mk(v[k].re * inv, v[k].im * inv);
            st_sp_site<double, S>(f.p + base + (int64_t)d * 12 * Vd, s, Vd, y);
        } else {
            for (int k = 0; k < 12; k++) st_c<double>(p + (int64_t)k * Vd, mk(v[k].re * inv, v[k].im * inv));
        }
    } else {
        for (int k = 0; k < 12; k++) st_c<double>(p + (int64_t)k * Vd, v[k]);
    }
}

template <typename S>
__device__ __forceinline__ void load_spinor_d(Field<S> f, int64_t base, int64_t sbase, int Vd, int d, int s,
                                              cpx<double> *v)
{
    if constexpr (S::kQuad) {
        double sc = (double)f.scale[sbase + (int64_t)d * Vd + s];
        ld_sp_site<double, S>(f.p + base + (int64_t)d * 12 * Vd, s, Vd, v);
        for (int k = 0; k < 12; k++) v[k] = sc * v[k];
    } else {
        const typename S::T2 *p = f.p + base + (int64_t)d * 12 * Vd + s;
        double sc = S::kScaled ? (double)f.scale[sbase + (int64_t)d * Vd + s] : 1.0;
        for (int k = 0; k < 12; k++) v[k] = sc * ld_c<double>(p + (int64_t)k * Vd);
    }
}

__global__ void k_links_in(Geom g, const int *site_of, const double2 *src, double2 *dst)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int d, s;
    split_index(g, gi, d, s);
    const double2 *p = src + (int64_t)__ldg(site_of + gi) * 36;
    for (int k = 0; k < 36; k++) dst[((int64_t)d * 36 + k) * g.Vd + s] = __ldg(p + k);
}

template <typename S>
__global__ void k_spinor_in(Geom g, const int *site_of, const double2 *src, Field<S> dst, int64_t rstride,
                            int64_t sstride)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int r = blockIdx.y;
    int d, s;
    split_index(g, gi, d, s);
    const double2 *p = src + ((int64_t)r * g.V + __ldg(site_of + gi)) * 12;
    cpx<double> v[12];
    for (int k = 0; k < 12; k++) {
        double2 a = __ldg(p + k);
        v[k] = mk(a.x, a.y);
    }
    store_spinor<S>(dst, r * rstride, r * sstride, g.Vd, d, s, v);
}

template <typename S>
__global__ void k_spinor_out(Geom g, const int *site_of, Field<S> src, int64_t rstride, int64_t sstride,
                             double2 *dst)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int r = blockIdx.y;
    int d, s;
    split_index(g, gi, d, s);
    cpx<double> v[12];
    load_spinor_d<S>(src, r * rstride, r * sstride, g.Vd, d, s, v);
    double2 *p = dst + ((int64_t)r * g.V + __ldg(site_of + gi)) * 12;
    for (int k = 0; k < 12; k++) p[k] = make_double2(v[k].re, v[k].im);
}

template <typename SI, typename SO>
__global__ void k_spinor_convert(Geom g, Field<SI> src, Field<SO> dst, int64_t rstride, int64_t sstride)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int r = blockIdx.y;
    int d, s;
    split_index(g, gi, d, s);
    cpx<double> v[12];
    load_spinor_d<SI>(src, r * rstride, r * sstride, g.Vd, d, s, v);
    store_spinor<SO>(dst, r * rstride, r * sstride, g.Vd, d, s, v);
}

// v = w / |w| in FP64 (out64, may alias w; |w|^2 from the device) and the
// same vector in a 16-bit storage with its per-site scale, in one pass: the
// Arnoldi step's new basis vector and the Schwarz input made from it.  The
// scaling is the FP64 arithmetic of the plain scaling kernel; the 16-bit copy
// is rounded from the FP32 value.  One thread per site.
template <typename SO>
__global__ void k_scale_convert(Geom g, const double2 *w, const double2 *norm2, double2 *out64, Field<SO> dst)
{
    __shared__ double fs;  // once per block: FP64 square root and division are long on the FP64 pipe
    if (threadIdx.x == 0) {
        double nn = norm2[0].x;
        fs = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int d, s;
    split_index(g, gi, d, s);
    const double f = fs;
    const int64_t base = (int64_t)d * 12 * g.Vd + s;
    cpx<float> v[12];
    float m = 0.f;
    for (int k = 0; k < 12; k++) {
        double2 a = w[base + (int64_t)k * g.Vd];
        a = make_double2(a.x * f, a.y * f);
        out64[base + (int64_t)k * g.Vd] = a;
        v[k] = mk((float)a.x, (float)a.y);
        m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
    }
    dst.scale[(int64_t)d * g.Vd + s] = m;
    const float inv = m > 0.f ? 1.f / m : 0.f;
    if constexpr (SO::kQuad) {
        for (int k = 0; k < 12; k++) v[k] = inv * v[k];
        st_sp_site<float, SO>(dst.p + (int64_t)d * 12 * g.Vd, s, g.Vd, v);
    } else {
        typename SO::T2 *p = dst.p + base;
        for (int k = 0; k < 12; k++) st_c<float>(p + (int64_t)k * g.Vd, inv * v[k]);
    }
}

template <typename S>
__global__ void k_links_convert(int64_t n, const double2 *src, typename S::T2 *dst)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = __ldg(src + i);
    st_c<double>(dst + i, mk(a.x, a.y));
}

// FP64 complex -> (re.hi, re.lo, im.hi, im.lo) FP32 split
__global__ void k_split_convert(int64_t n, const double2 *src, float4 *dst)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = __ldg(src + i);
    float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
    dst[i] = make_float4(rh, __double2float_rn(a.x - (double)rh), ih, __double2float_rn(a.y - (double)ih));
}

// Sets *bad when a link is not SU(3) to tol: max |(U U^+ - 1)_ij| or |det U - 1|.
// One thread per link (domain d, direction mu, site s).
__global__ void k_su3_check(Geom g, const double2 *U, double tol, int *bad)
{
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= (int64_t)g.V * 4) return;
    const int64_t d = li / (4 * g.Vd);
    const int mu = (int)((li / g.Vd) % 4), s = (int)(li % g.Vd);
    const double2 *p = U + (d * 36 + mu * 9) * g.Vd + s;
    cpx<double> u[9];
    for (int k = 0; k < 9; k++) {
        double2 a = __ldg(p + (int64_t)k * g.Vd);
        u[k] = mk(a.x, a.y);
    }
    double dev = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cpx<double> t = mk(i == j ? -1.0 : 0.0, 0.0);
            for (int k = 0; k < 3; k++) t = t + u[i * 3 + k] * conj(u[j * 3 + k]);
            dev = fmax(dev, fmax(fabs(t.re), fabs(t.im)));
        }
    cpx<double> det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                      u[2] * (u[3] * u[7] - u[4] * u[6]);
    dev = fmax(dev, fmax(fabs(det.re - 1.0), fabs(det.im)));
    if (!(dev <= tol)) atomicOr(bad, 1);
}

// The first two rows of every link: 24 planes per site, plane mu*6 + 3*row + col
// (an SU(3) link's third row is the conjugated cross product of the two).
// 16-bit formats are stored with planes paired (pair_index below), so that
// the operator reads two planes with one 8-byte load.
template <typename S>
__global__ void k_links12_convert(Geom g, const double2 *src, typename S::T2 *dst)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int d, s;
    split_index(g, gi, d, s);
    for (int mu = 0; mu < 4; mu++)
        for (int k = 0; k < 6; k++) {
            double2 a = __ldg(src + ((int64_t)d * 36 + mu * 9 + k) * g.Vd + s);
            const int p = mu * 6 + k;
            st_c<double>(dst + (S::kBytes == 4 ? pair_index(d, 24, p, g.Vd, s) : ((int64_t)d * 24 + p) * g.Vd + s),
                         mk(a.x, a.y));
        }
}

// clover blocks: 36 planes per site; 16-bit formats get one scale per site
// (paired: planes stored in pairs, for the full-lattice operator's copy)
template <typename S>
__global__ void k_clover_convert(Geom g, const double2 *src, Field<S> dst, int paired)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int d, s;
    split_index(g, gi, d, s);
    const double2 *p = src + (int64_t)d * 36 * g.Vd + s;
    typename S::T2 *q = dst.p + (int64_t)d * 36 * g.Vd + s;
    double inv = 1.0;
    if (S::kScaled) {
        double m = 0;
        for (int k = 0; k < 36; k++) {
            double2 a = __ldg(p + (int64_t)k * g.Vd);
            m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
        }
        float sc = (float)m;
        dst.scale[gi] = sc;
        inv = m > 0 ? 1.0 / (double)sc : 0.0;
    }
    for (int k = 0; k < 36; k++) {
        double2 a = __ldg(p + (int64_t)k * g.Vd);
        typename S::T2 *o = paired ? dst.p + pair_index(d, 36, k, g.Vd, s) : q + (int64_t)k * g.Vd;
        st_c<double>(o, mk(a.x * inv, a.y * inv));
    }
}

// -------------------------------------------------------------- launchers

static inline dim3 grid_sites(int V, int nrhs, int bs) { return dim3((V + bs - 1) / bs, nrhs); }

qdd_status launch_links_to_internal(Gauge *g, const double *src, cudaStream_t s)
{
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    k_links_in<<<grid_sites(g->hg.V, 1, 256), 256, 0, s>>>(g->geom, g->d_site_of.as<int>(), (const double2 *)src,
                                                           g->links64.as<double2>());
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

#define QDD_DISPATCH_PREC(prec, S, ...)                   \
    switch (prec) {                                       \
    case QDD_PREC_F64: { using S = StF64; __VA_ARGS__; break; } \
    case QDD_PREC_F32: { using S = StF32; __VA_ARGS__; break; } \
    case QDD_PREC_F16S: { using S = StF16; __VA_ARGS__; break; } \
    case QDD_PREC_BF16S: { using S = StBF16; __VA_ARGS__; break; } \
    default: set_error("invalid precision %d", (int)prec); return QDD_EINVAL; \
    }

qdd_status launch_spinor_in(Gauge *g, const double *src, void *dst, float *dst_scale, qdd_prec prec, int nrhs,
                            cudaStream_t s)
{
    const HostGeom &hg = g->hg;
    int64_t rs = (int64_t)hg.V * 12, ss = hg.V;
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(prec, S, {
        Field<S> f{(typename S::T2 *)dst, dst_scale};
        k_spinor_in<S><<<grid_sites(hg.V, nrhs, 256), 256, 0, s>>>(g->geom, g->d_site_of.as<int>(),
                                                                   (const double2 *)src, f, rs, ss);
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_spinor_out(Gauge *g, const void *src, const float *src_scale, double *dst, qdd_prec prec, int nrhs,
                             cudaStream_t s)
{
    const HostGeom &hg = g->hg;
    int64_t rs = (int64_t)hg.V * 12, ss = hg.V;
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(prec, S, {
        Field<S> f{(typename S::T2 *)src, (float *)src_scale};
        k_spinor_out<S><<<grid_sites(hg.V, nrhs, 256), 256, 0, s>>>(g->geom, g->d_site_of.as<int>(), f, rs, ss,
                                                                    (double2 *)dst);
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_spinor_convert(Gauge *g, const void *src, const float *src_scale, qdd_prec sp, void *dst,
                                 float *dst_scale, qdd_prec dp, int nrhs, cudaStream_t s)
{
    const HostGeom &hg = g->hg;
    int64_t rs = (int64_t)hg.V * 12, ss = hg.V;
    dim3 grid = grid_sites(hg.V, nrhs, 256);
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(sp, SI, {
        Field<SI> fi{(typename SI::T2 *)src, (float *)src_scale};
        QDD_DISPATCH_PREC(dp, SO, {
            Field<SO> fo{(typename SO::T2 *)dst, dst_scale};
            k_spinor_convert<SI, SO><<<grid, 256, 0, s>>>(g->geom, fi, fo, rs, ss);
        });
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_scale_convert(Gauge *g, const double2 *w, const double2 *norm2, double2 *out64, void *dst,
                                float *dst_scale, qdd_prec dp, cudaStream_t s)
{
    const int64_t n = (int64_t)g->hg.V * 12;
    g->ctx->timer.work(K_BLAS, 2.0 * n, (32.0 + 4.0) * n + 4.0 * g->hg.V);
    LaunchScope ls(g->ctx->timer, K_BLAS, s);
    const unsigned grid = (unsigned)((g->hg.V + 127) / 128);
    if (dp == QDD_PREC_F16S)
        k_scale_convert<StF16><<<grid, 128, 0, s>>>(g->geom, w, norm2, out64, Field<StF16>{(__half2 *)dst, dst_scale});
    else if (dp == QDD_PREC_BF16S)
        k_scale_convert<StBF16><<<grid, 128, 0, s>>>(g->geom, w, norm2, out64,
                                                     Field<StBF16>{(__nv_bfloat162 *)dst, dst_scale});
    else {
        set_error("scale-and-convert takes a 16-bit storage");
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_links_convert(Gauge *g, qdd_prec dp, void *dst, cudaStream_t s)
{
    int64_t n = (int64_t)g->hg.V * 36;
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(dp, S, {
        k_links_convert<S><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, g->links64.as<double2>(),
                                                                        (typename S::T2 *)dst);
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_su3_check(Gauge *g, double tol, int *d_bad, cudaStream_t s)
{
    const int64_t n = (int64_t)g->hg.V * 4;
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    k_su3_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->geom, g->links64.as<double2>(), tol, d_bad);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_links12_convert(Gauge *g, qdd_prec dp, void *dst, cudaStream_t s)
{
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(dp, S, {
        k_links12_convert<S><<<grid_sites(g->hg.V, 1, 256), 256, 0, s>>>(g->geom, g->links64.as<double2>(),
                                                                          (typename S::T2 *)dst);
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_split_convert(Gauge *g, const double2 *src, float4 *dst, int64_t n, cudaStream_t s)
{
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    k_split_convert<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, src, dst);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

qdd_status launch_clover_convert(Gauge *g, const double2 *src, qdd_prec dp, void *dst, float *dst_scale,
                                 cudaStream_t s, bool paired)
{
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    QDD_DISPATCH_PREC(dp, S, {
        Field<S> f{(typename S::T2 *)dst, dst_scale};
        k_clover_convert<S><<<grid_sites(g->hg.V, 1, 256), 256, 0, s>>>(g->geom, src, f,
                                                                         paired && S::kBytes == 4 ? 1 : 0);
    });
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

}  // namespace qdd
