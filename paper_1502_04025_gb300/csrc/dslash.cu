// Full-lattice Wilson-clover operator  y = D x = A x - kappa H x
// (arXiv:1502.04025, Sec. 3.1 names the operator; Sec. 3.6 counts 1848 flop
// per site: 1320 for the eight spin-projected hops, 504 for the two Hermitian
// 6x6 clover blocks, 24 for the final combination).
//
// One thread per site over the domain-blocked, plane-major layout: a warp
// reads 32 consecutive sites of one plane (256 or 512 contiguous bytes) for
// every link, clover and spinor component.  Domains are visited in
// lexicographic block order, so a domain's neighbours are processed close in
// time and their spinors are read from L2 rather than again from HBM.  Neighbour sites come from a
// per-domain-shape table (the neighbour's slot inside its domain and whether
// the hop leaves the domain) and a per-domain table of neighbouring domains.
// The roofline of this kernel is HBM bandwidth: each link, clover entry and
// input spinor is read once and the output written once when the neighbour
// re-reads hit in L1/L2.  For SU(3) fields the FP32 and 16-bit forms read
// only the first two rows of each link and rebuild the third (96 fewer bytes
// per site in FP32), and their 16-bit link and clover copies are stored with
// planes paired, one 8-byte load per two planes.
#include <type_traits>

#include "internal.h"

namespace qdd {

// FP16 spinors (quad planes): site s of the domain block at blk_base, scaled
template <typename R, typename S>
__device__ __forceinline__ void load_spinor_quad(const Field<S> &f, int64_t blk_base, int s, int64_t sidx, int Vd,
                                                 cpx<R> *x)
{
    const R sc = (R)__ldg(f.scale + sidx);
    ld_sp_site<R, S>(f.p + blk_base, s, Vd, x);
#pragma unroll
    for (int k = 0; k < 12; k++) x[k] = sc * x[k];
}

// spinors in planes: the site's first component at gi_plane_base
template <typename R, typename S>
__device__ __forceinline__ void load_spinor(const Field<S> &f, int64_t gi_plane_base, int64_t sidx, int Vd,
                                            cpx<R> *x)
{
    const typename S::T2 *p = f.p + gi_plane_base;
    R sc = S::kScaled ? (R)__ldg(f.scale + sidx) : (R)1;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        cpx<R> v = ld_c<R>(p + (int64_t)k * Vd);
        x[k] = S::kScaled ? sc * v : v;
    }
}

// Two adjacent planes of a paired 16-bit field with one 8-byte load.
template <typename R>
__device__ __forceinline__ void ld_pair(const __half2 *p, cpx<R> &a, cpx<R> &b)
{
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    a = mk<R>(f0.x, f0.y);
    b = mk<R>(f1.x, f1.y);
}
template <typename R>
__device__ __forceinline__ void ld_pair(const __nv_bfloat162 *p, cpx<R> &a, cpx<R> &b)
{
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    a = mk<R>(f0.x, f0.y);
    b = mk<R>(f1.x, f1.y);
}

// Link U_mu of site s of domain d.  L12: the field holds the first two rows
// (24 planes per site) and the third is rebuilt as the conjugated cross
// product of the two, i.e. from the cofactors of U = (U^+)^-1 for det U = 1.
template <typename R, typename S, bool L12>
__device__ __forceinline__ void load_link(const Field<S> &U, int d, int s, int mu, int Vd, cpx<R> *u)
{
    if (L12) {
        if constexpr (S::kBytes == 4) {  // 16-bit: paired planes
            const typename S::T2 *p = U.p + pair_index(d, 24, mu * 6, Vd, s);
#pragma unroll
            for (int j = 0; j < 3; j++) ld_pair<R>(p + (int64_t)j * Vd * 2, u[2 * j], u[2 * j + 1]);
        } else {
            const typename S::T2 *p = U.p + ((int64_t)d * 24 + mu * 6) * Vd + s;
#pragma unroll
            for (int k = 0; k < 6; k++) u[k] = ld_c<R>(p + (int64_t)k * Vd);
        }
        u[6] = conj(u[1] * u[5] - u[2] * u[4]);
        u[7] = conj(u[2] * u[3] - u[0] * u[5]);
        u[8] = conj(u[0] * u[4] - u[1] * u[3]);
    } else {
        const typename S::T2 *p = U.p + ((int64_t)d * 36 + mu * 9) * Vd + s;
#pragma unroll
        for (int k = 0; k < 9; k++) u[k] = ld_c<R>(p + (int64_t)k * Vd);
    }
}

// one hop of a neighbour spinor x stored with per-site scale sc: the hop is
// linear, so the scale multiplies its 6-component result, not the 12 inputs
template <int MU, int SGN, bool SCALED, bool PAIRED, typename R>
__device__ __forceinline__ void hop_scaled(const cpx<R> *U, const cpx<R> *x, R sc, cpx<R> *acc)
{
    cpx<R> h[6], w[6];
    project<MU, SGN>(x, h);
    su3_mul_half<(SGN < 0), R, PAIRED>(U, h, w);
    if (SCALED) {
#pragma unroll
        for (int k = 0; k < 6; k++) w[k] = sc * w[k];
    }
    reconstruct_add<MU, SGN>(w, acc);
}

// the unscaled components of a spinor and, for a 16-bit field, its scale;
// fields in planes: the site's first component at gi_plane_base; FP16 fields
// (quad planes): site s of the domain block at blk_base
template <typename R, typename S>
__device__ __forceinline__ R load_spinor_raw_quad(const Field<S> &f, int64_t blk_base, int s, int64_t sidx, int Vd,
                                                  cpx<R> *x)
{
    ld_sp_site<R, S>(f.p + blk_base, s, Vd, x);
    return (R)__ldg(f.scale + sidx);
}

template <typename R, typename S>
__device__ __forceinline__ R load_spinor_raw(const Field<S> &f, int64_t gi_plane_base, int64_t sidx, int Vd,
                                             cpx<R> *x)
{
    const typename S::T2 *p = f.p + gi_plane_base;
#pragma unroll
    for (int k = 0; k < 12; k++) x[k] = ld_c<R>(p + (int64_t)k * Vd);
    return S::kScaled ? (R)__ldg(f.scale + sidx) : (R)1;
}

template <int MU, typename R, typename SL, typename SI, bool L12>
__device__ __forceinline__ void dslash_dir(const Geom &g, const Field<SL> &U, const Field<SI> &in, int64_t rbase,
                                           int64_t sbase, int d, int s, cpx<R> *acc)
{
    // paired FMAs in the colour products, except with FP16 links and FP32
    // spinors, where they measured slower (192.7 against 200.7 us on 32^3x64)
    constexpr bool kPaired = !(std::is_same<SL, StF16>::value && std::is_same<SI, StF32>::value);
    cpx<R> u[9], x[12];
    {
        uint16_t e = __ldg(g.nbl + s * 8 + 2 * MU);
        int nd = (e & kCross) ? __ldg(g.nbd + d * 8 + 2 * MU) : d;
        int ns = e & kSlotMask;
        if (QDD_IN_RANGE(nd, 0, g.Nd) && QDD_IN_RANGE(ns, 0, g.Vd)) {
            R sc;
            if constexpr (SI::kQuad)
                sc = load_spinor_raw_quad<R, SI>(in, rbase + (int64_t)nd * 12 * g.Vd, ns,
                                                 sbase + (int64_t)nd * g.Vd + ns, g.Vd, x);
            else
                sc = load_spinor_raw<R, SI>(in, rbase + (int64_t)nd * 12 * g.Vd + ns, sbase + (int64_t)nd * g.Vd + ns,
                                            g.Vd, x);
            load_link<R, SL, L12>(U, d, s, MU, g.Vd, u);
            hop_scaled<MU, +1, SI::kScaled, kPaired>(u, x, sc, acc);
        }
    }
    {
        uint16_t e = __ldg(g.nbl + s * 8 + 2 * MU + 1);
        int nd = (e & kCross) ? __ldg(g.nbd + d * 8 + 2 * MU + 1) : d;
        int ns = e & kSlotMask;
        if (QDD_IN_RANGE(nd, 0, g.Nd) && QDD_IN_RANGE(ns, 0, g.Vd)) {
            R sc;
            if constexpr (SI::kQuad)
                sc = load_spinor_raw_quad<R, SI>(in, rbase + (int64_t)nd * 12 * g.Vd, ns,
                                                 sbase + (int64_t)nd * g.Vd + ns, g.Vd, x);
            else
                sc = load_spinor_raw<R, SI>(in, rbase + (int64_t)nd * 12 * g.Vd + ns, sbase + (int64_t)nd * g.Vd + ns,
                                            g.Vd, x);
            load_link<R, SL, L12>(U, nd, ns, MU, g.Vd, u);
            hop_scaled<MU, -1, SI::kScaled, kPaired>(u, x, sc, acc);
        }
    }
}

// The geometry with the domain volume fixed at compile time when VD > 0 (a
// power of two): plane strides and site splits become immediates.
template <int VD>
__device__ __forceinline__ Geom fixed_geom(const Geom &g0)
{
    Geom g = g0;
    if (VD > 0) {
        static_assert(VD <= 0 || (VD & (VD - 1)) == 0, "a fixed domain volume is a power of two");
        g.Vd = VD;
        g.Vh = VD / 2;
        g.vd_shift = VD == 256 ? 8 : (VD == 512 ? 9 : (VD == 128 ? 7 : g0.vd_shift));
    }
    return g;
}

// CTAs per SM the register allocation aims at.  FP16 links: 4 (the lower
// register cap of 5 costs more in the FP16 and H16 forms: on 32^3x64, FP16
// 181.5 -> 175.0 us and H16 193.6 -> 190.1 us at 4; FP32 and BF16 are
// faster at 5, BF16 176.6 against 188.0 us).
template <typename R, typename SL>
constexpr int dslash_min_blocks()
{
    return sizeof(R) == 4 ? (std::is_same<SL, StF16>::value ? 4 : 5) : 1;
}

template <typename R, typename SL, typename SC, typename SI, typename SO, bool RESID, bool L12, int VD = 0>
__global__ void __launch_bounds__(128, (dslash_min_blocks<R, SL>())) k_dslash(Geom g0, Field<SL> U, Field<SC> A, Field<SI> in, Field<SO> out,
                                                const double2 *b, R kappa)
{
    const Geom g = fixed_geom<VD>(g0);
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    const int64_t r = blockIdx.y;
    const int64_t rbase = r * (int64_t)g.V * 12, sbase = r * (int64_t)g.V;
    int d, s;
    lex_site(g, gi, d, s);
    gi = d * g.Vd + s;
    cpx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
    dslash_dir<0, R, SL, SI, L12>(g, U, in, rbase, sbase, d, s, acc);
    dslash_dir<1, R, SL, SI, L12>(g, U, in, rbase, sbase, d, s, acc);
    dslash_dir<2, R, SL, SI, L12>(g, U, in, rbase, sbase, d, s, acc);
    dslash_dir<3, R, SL, SI, L12>(g, U, in, rbase, sbase, d, s, acc);

    cpx<R> x[12];
    if constexpr (SI::kQuad)
        load_spinor_quad<R, SI>(in, rbase + (int64_t)d * 12 * g.Vd, s, sbase + gi, g.Vd, x);
    else
        load_spinor<R, SI>(in, rbase + (int64_t)d * 12 * g.Vd + s, sbase + gi, g.Vd, x);
    cpx<R> y[12];
    {
        const typename SC::T2 *p = A.p + (int64_t)d * 36 * g.Vd + s;
        R sc = SC::kScaled ? (R)__ldg(A.scale + gi) : (R)1;
        cpx<R> m[2][18];
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            if constexpr (SC::kBytes == 4) {  // 16-bit: paired planes
                const typename SC::T2 *pp = A.p + pair_index(d, 36, blk * 18, g.Vd, s);
#pragma unroll
                for (int j = 0; j < 9; j++) ld_pair<R>(pp + (int64_t)j * g.Vd * 2, m[blk][2 * j], m[blk][2 * j + 1]);
            } else {
#pragma unroll
                for (int k = 0; k < 18; k++) m[blk][k] = ld_c<R>(p + (int64_t)(blk * 18 + k) * g.Vd);
            }
        }
        // The two blocks as paired FMAs (the same bits) only with FP16 clover and
        // spinors: 175.0 -> 171.9 us on 32^3x64.  Measured slower in the other
        // forms: FP32 256.7 -> 344.0 us at 96 registers, H16 190.1 -> 198.2 us.
        if constexpr (std::is_same<SC, StF16>::value && std::is_same<SI, StF16>::value) {
            herm6_mul_x2(m[0], m[1], x, y);
        } else {
            herm6_mul(m[0], x, y);
            herm6_mul(m[1], x + 6, y + 6);
        }
        if (SC::kScaled) {  // the clover's per-site scale on the 12 products
#pragma unroll
            for (int k = 0; k < 12; k++) y[k] = sc * y[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 12; k++) {
        y[k].re = fma(-kappa, acc[k].re, y[k].re);
        y[k].im = fma(-kappa, acc[k].im, y[k].im);
    }
    if (RESID) {
        const double2 *bp = b + rbase + (int64_t)d * 12 * g.Vd + s;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 v = __ldg(bp + (int64_t)k * g.Vd);
            y[k] = mk<R>((R)v.x - y[k].re, (R)v.y - y[k].im);
        }
    }
    typename SO::T2 *op = out.p + rbase + (int64_t)d * 12 * g.Vd + s;
    if (SO::kScaled) {
        R m = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) m = fmax(m, fmax(fabs(y[k].re), fabs(y[k].im)));
        float scf = (float)m;
        out.scale[sbase + gi] = scf;
        R inv = m > 0 ? (R)1 / (R)scf : (R)0;
        if constexpr (SO::kQuad) {
#pragma unroll
            for (int k = 0; k < 12; k++) y[k] = inv * y[k];
            st_sp_site<R, SO>(out.p + rbase + (int64_t)d * 12 * g.Vd, s, g.Vd, y);
        } else {
#pragma unroll
            for (int k = 0; k < 12; k++) st_c<R>(op + (int64_t)k * g.Vd, inv * y[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 12; k++) st_c<R>(op + (int64_t)k * g.Vd, y[k]);
    }
}

// ------------------------------------------------------------------------
// Double-float operator: y = D x with every product and sum carried as a pair
// of FP32 numbers (error-free transformations), from links and clover split
// into hi + lo FP32 parts.  About 2^-46 relative accuracy at a fraction of the
// cost of FP64 arithmetic on this GPU; used for w = D z_j in the Arnoldi step.

__device__ __forceinline__ cdf ld_cdf(const float4 *p)
{
    float4 v = __ldg(p);
    return {{v.x, v.y}, {v.z, v.w}};
}

__device__ __forceinline__ cdf ld_in_df(const float2 *p)
{
    float2 v = __ldg(p);
    return {{v.x, 0.f}, {v.y, 0.f}};
}

__device__ __forceinline__ cdf ld_in_df(const double2 *p)
{
    double2 v = __ldg(p);
    return {df_from_double(v.x), df_from_double(v.y)};
}

// Spin structure of one hop in the chiral basis.  With u the upper and l the
// lower two spins, (1 -+ gamma_mu) x projects to h = u -+ A l and the lower
// spins of the result are -+ A^dagger (U h), where A is a 2x2 matrix of unit
// complex numbers, anti-diagonal for x, y and diagonal for z, t:
//   x: A = [[0, -i], [-i, 0]]   y: A = [[0, -1], [1, 0]]
//   z: A = [[-i, 0], [0, i]]    t: A = 1
// One direction and sign is therefore a swap flag, a rotate-by-i flag and
// four signs.  The double-float operator runs one hop body driven by these
// runtime values: eight inlined copies of its long double-float chains did
// not fit the instruction cache.
struct HopSpin {
    bool swap, rot;
    float p0, p1;  // h_0 = u_0 + p0 (rot ? i : 1) l_{swap}, h_1 = u_1 + p1 (rot ? i : 1) l_{1-swap}
    float r0, r1;  // lower_0 += r0 (rot ? i : 1) w_{swap}, lower_1 += r1 (rot ? i : 1) w_{1-swap}
};

__device__ __forceinline__ HopSpin hop_spin(int mu, int back)
{
    const bool swap = mu < 2, rot = (mu & 1) == 0;
    const float s0 = mu == 3 ? 1.f : -1.f;  // A's row-0 entry = s0 (rot ? i : 1)
    const float s1 = mu == 0 ? -1.f : 1.f;  // A's row-1 entry = s1 (rot ? i : 1)
    const float t = back ? 1.f : -1.f;      // forward hop: h = u - A l; backward: h = u + A l
    // rows of A^dagger: conjugate transpose; conjugation flips an imaginary unit
    float d0 = swap ? s1 : s0, d1 = swap ? s0 : s1;
    if (rot) {
        d0 = -d0;
        d1 = -d1;
    }
    return {swap, rot, t * s0, t * s1, t * d0, t * d1};
}

// sg * (rot ? i z : z), exact
__device__ __forceinline__ cdf cdf_unit(bool rot, float sg, cdf z)
{
    df a = rot ? df_neg(z.im) : z.re;
    df b = rot ? z.re : z.im;
    return {{__fmul_rn(sg, a.hi), __fmul_rn(sg, a.lo)}, {__fmul_rn(sg, b.hi), __fmul_rn(sg, b.lo)}};
}

__device__ __forceinline__ cdf cdf_sel(bool c, cdf a, cdf b) { return c ? a : b; }

// Two double-float multiply-accumulates at once, as the two lanes of paired
// FP32 operations: each lane runs dfacc_mul_add's sequence of operations
// (TwoProd by FMA, TwoSum, the error terms summed in the same order), so
// each lane's result is the same bits as the scalar form.  Used for the two
// spins of a half spinor, which share every link entry.
struct dfacc2 {
    float2 s, c;
};

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

__device__ __forceinline__ void dfacc2_mul_add(dfacc2 &acc, df x, float2 yhi, float2 ylo)
{
    const float2 xh = bc2(x.hi), xl = bc2(x.lo);
    const float2 p = __fmul2_rn(xh, yhi);
    float2 e = __ffma2_rn(xh, yhi, neg2(p));
    e = __ffma2_rn(xh, ylo, e);
    e = __ffma2_rn(xl, yhi, e);
    // TwoSum(acc.s, p)
    const float2 s = __fadd2_rn(acc.s, p);
    const float2 bb = __fadd2_rn(s, neg2(acc.s));
    const float2 t = __fadd2_rn(__fadd2_rn(acc.s, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
    acc.s = s;
    acc.c = __fadd2_rn(acc.c, __fadd2_rn(t, e));
}

// value of the pair's two accumulators (FastTwoSum per lane)
__device__ __forceinline__ void dfacc2_value(const dfacc2 &a, df &v0, df &v1)
{
    const float2 s = __fadd2_rn(a.s, a.c);
    const float2 e = __fadd2_rn(a.c, neg2(__fadd2_rn(s, neg2(a.s))));
    v0 = {s.x, e.x};
    v1 = {s.y, e.y};
}

// w = U h for both spins of the half spinor h (row-major U, the oriented
// link), the two spins as the lanes of paired operations
__device__ __forceinline__ void su3_mul_half_df2(const cdf *U, const cdf *h, cdf *w)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        dfacc2 re = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        dfacc2 im = re;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const cdf u = U[a * 3 + b];
            const cdf h0 = h[b], h1 = h[3 + b];
            const float2 rhi = make_float2(h0.re.hi, h1.re.hi), rlo = make_float2(h0.re.lo, h1.re.lo);
            const float2 ihi = make_float2(h0.im.hi, h1.im.hi), ilo = make_float2(h0.im.lo, h1.im.lo);
            // cdfacc_mul_add<false>: re += u.re h.re, re += (-u.im) h.im, im += u.re h.im, im += u.im h.re
            dfacc2_mul_add(re, u.re, rhi, rlo);
            dfacc2_mul_add(re, df_neg(u.im), ihi, ilo);
            dfacc2_mul_add(im, u.re, ihi, ilo);
            dfacc2_mul_add(im, u.im, rhi, rlo);
        }
        df r0, r1, i0, i1;
        dfacc2_value(re, r0, r1);
        dfacc2_value(im, i0, i1);
        w[a] = {r0, i0};
        w[3 + a] = {r1, i1};
    }
}

// the double-float colour products with the two spins as paired lanes (the
// 48^3x96 solve's operator class 44.41 -> 43.56 ms, the same solution bits)
constexpr bool kPairedDf = true;

// acc += hop contribution; U is the oriented link (U(n) for a forward hop,
// U(n - mu)^dagger for a backward one), row-major
__device__ __forceinline__ void hop_df_rt(const HopSpin &hs, const cdf *U, const cdf *x, cdfacc *acc)
{
    cdf h[6];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cdf l0 = x[6 + c], l1 = x[9 + c];
        h[c] = cdf_add(x[c], cdf_unit(hs.rot, hs.p0, cdf_sel(hs.swap, l1, l0)));
        h[3 + c] = cdf_add(x[3 + c], cdf_unit(hs.rot, hs.p1, cdf_sel(hs.swap, l0, l1)));
    }
    cdf w[6];
    if constexpr (kPairedDf) {
        su3_mul_half_df2(U, h, w);
    } else {
#pragma unroll
        for (int sp = 0; sp < 2; sp++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                cdfacc t;
                cdfacc_zero(t);
#pragma unroll
                for (int b = 0; b < 3; b++) cdfacc_mul_add<false>(t, U[a * 3 + b], h[sp * 3 + b]);
                w[sp * 3 + a] = cdfacc_value(t);
            }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cdf w0 = w[c], w1 = w[3 + c];
        cdf b0 = cdf_unit(hs.rot, hs.r0, cdf_sel(hs.swap, w1, w0));
        cdf b1 = cdf_unit(hs.rot, hs.r1, cdf_sel(hs.swap, w0, w1));
        dfacc_add(acc[0 * 3 + c].re, w0.re); dfacc_add(acc[0 * 3 + c].im, w0.im);
        dfacc_add(acc[1 * 3 + c].re, w1.re); dfacc_add(acc[1 * 3 + c].im, w1.im);
        dfacc_add(acc[2 * 3 + c].re, b0.re); dfacc_add(acc[2 * 3 + c].im, b0.im);
        dfacc_add(acc[3 * 3 + c].re, b1.re); dfacc_add(acc[3 * 3 + c].im, b1.im);
    }
}

template <typename SI, int VD = 0>
__global__ void __launch_bounds__(128, 4) k_dslash_df(Geom g0, const float4 *U, const float4 *A,
                                                   const typename SI::T2 *in, double2 *out, df kappa)
{
    const Geom g = fixed_geom<VD>(g0);
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    const int64_t rbase = (int64_t)blockIdx.y * g.V * 12;
    int d, s;
    lex_site(g, gi, d, s);
    cdfacc acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) cdfacc_zero(acc[k]);
#pragma unroll 1
    for (int dir = 0; dir < 8; dir++) {
        const int mu = dir >> 1, back = dir & 1;
        uint16_t e = __ldg(g.nbl + s * 8 + dir);
        int nd = (e & kCross) ? __ldg(g.nbd + d * 8 + dir) : d;
        int ns = e & kSlotMask;
        if (!(QDD_IN_RANGE(nd, 0, g.Nd) && QDD_IN_RANGE(ns, 0, g.Vd))) continue;
        cdf x[12], u[9];
        const typename SI::T2 *xp = in + rbase + (int64_t)nd * 12 * g.Vd + ns;
#pragma unroll
        for (int k = 0; k < 12; k++) x[k] = ld_in_df(xp + (int64_t)k * g.Vd);
        const int ld = back ? nd : d, ls = back ? ns : s;
        const float4 *up = U + ((int64_t)ld * 36 + mu * 9) * g.Vd + ls;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            // backward hop: element (a, b) of U^dagger is conj(U_ba)
            const int src = back ? (k % 3) * 3 + k / 3 : k;
            cdf v = ld_cdf(up + (int64_t)src * g.Vd);
            u[k] = back ? cdf{v.re, df_neg(v.im)} : v;
        }
        hop_df_rt(hop_spin(mu, back), u, x, acc);
    }
    // y = A x - kappa * (hop sum), one chirality block per iteration; the
    // block's hop sum is always hv[0..5] (the second block is shifted down)
    cdf hv[12];
#pragma unroll
    for (int k = 0; k < 12; k++) hv[k] = cdfacc_value(acc[k]);
    const typename SI::T2 *xp = in + rbase + (int64_t)d * 12 * g.Vd + s;
    const float4 *ap = A + (int64_t)d * 36 * g.Vd + s;
    double2 *op = out + rbase + (int64_t)d * 12 * g.Vd + s;
    const df mk_ = df_neg(kappa);
#pragma unroll 1
    for (int blk = 0; blk < 2; blk++) {
        cdf x[6], m[18];
#pragma unroll
        for (int k = 0; k < 6; k++) x[k] = ld_in_df(xp + (int64_t)(6 * blk + k) * g.Vd);
#pragma unroll
        for (int k = 0; k < 18; k++) m[k] = ld_cdf(ap + (int64_t)(blk * 18 + k) * g.Vd);
        cdfacc y[6];
        df dg[6] = {m[0].re, m[0].im, m[1].re, m[1].im, m[2].re, m[2].im};
#pragma unroll
        for (int i = 0; i < 6; i++) {
            cdfacc_zero(y[i]);
            dfacc_mul_add(y[i].re, dg[i], x[i].re);
            dfacc_mul_add(y[i].im, dg[i], x[i].im);
        }
        int k = 3;
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = i + 1; j < 6; j++) {
                cdfacc_mul_add<false>(y[i], m[k], x[j]);
                cdfacc_mul_add<true>(y[j], m[k], x[i]);
                k++;
            }
#pragma unroll
        for (int i = 0; i < 6; i++) {
            dfacc_mul_add(y[i].re, mk_, hv[i].re);
            dfacc_mul_add(y[i].im, mk_, hv[i].im);
            cdf v = cdfacc_value(y[i]);
            op[(int64_t)(6 * blk + i) * g.Vd] = make_double2(df_to_double(v.re), df_to_double(v.im));
            hv[i] = hv[6 + i];
        }
    }
}

// out-of-range indices the kernels of this file have skipped (QDD_CHECK builds)
unsigned long long check_hits_dslash()
{
#ifdef QDD_CHECK
    unsigned long long h = 0;
    if (cudaMemcpyFromSymbol(&h, g_check_hits, sizeof(h)) != cudaSuccess) return ~0ull;
    return h;
#else
    return 0;
#endif
}

template <typename R, typename SL, typename SC, typename SI, typename SO, bool RESID, bool L12 = false>
static qdd_status run_dslash(Gauge *g, Field<SL> U, Field<SC> A, const void *in, const float *in_s, void *out,
                             float *out_s, const double2 *b, int nrhs, cudaStream_t s)
{
    Field<SI> fi{(typename SI::T2 *)in, (float *)in_s};
    Field<SO> fo{(typename SO::T2 *)out, out_s};
    dim3 grid((g->hg.V + 127) / 128, nrhs);
    LaunchScope ls(g->ctx->timer, K_DSLASH, s);
    if (g->hg.Vd == 256)  // 4^4 domains: the volume fixed at compile time
        k_dslash<R, SL, SC, SI, SO, RESID, L12, 256><<<grid, 128, 0, s>>>(g->geom, U, A, fi, fo, b, (R)g->kappa);
    else
        k_dslash<R, SL, SC, SI, SO, RESID, L12><<<grid, 128, 0, s>>>(g->geom, U, A, fi, fo, b, (R)g->kappa);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

// FP32 arithmetic on links of storage SL: the two-row copy when the gauge
// field allows it, else whole links
template <typename SL, typename SC, typename SI, typename SO>
static qdd_status run_dslash_lowp(Gauge *g, qdd_prec fp, Field<SC> A, const void *in, const float *in_s, void *out,
                                  float *out_s, int nrhs, cudaStream_t s)
{
    if (g->two_rows) {
        QDD_TRY(ensure_links12(g, fp, s));
        Field<SL> U{(typename SL::T2 *)g->copies[fp].links12.p, nullptr};
        return run_dslash<float, SL, SC, SI, SO, false, true>(g, U, A, in, in_s, out, out_s, nullptr, nrhs, s);
    }
    Field<SL> U{(typename SL::T2 *)g->copies[fp].links.p, nullptr};
    return run_dslash<float, SL, SC, SI, SO, false, false>(g, U, A, in, in_s, out, out_s, nullptr, nrhs, s);
}

qdd_status launch_dslash(Gauge *g, qdd_prec arith, qdd_prec fp, const void *in, const float *in_s, qdd_prec ip,
                         void *out, float *out_s, qdd_prec op, const double2 *b, int nrhs, cudaStream_t s)
{
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    if (arith == QDD_PREC_F64) {
        if (fp != QDD_PREC_F64 || op != QDD_PREC_F64) {
            set_error("FP64 operator needs FP64 fields and output");
            return QDD_EINVAL;
        }
        Field<StF64> U{g->links64.as<double2>(), nullptr}, A{g->clov64.as<double2>(), nullptr};
        switch (ip) {
        case QDD_PREC_F64:
            return b ? run_dslash<double, StF64, StF64, StF64, StF64, true>(g, U, A, in, in_s, out, out_s, b, nrhs, s)
                     : run_dslash<double, StF64, StF64, StF64, StF64, false>(g, U, A, in, in_s, out, out_s, b, nrhs,
                                                                             s);
        case QDD_PREC_F32:
            return run_dslash<double, StF64, StF64, StF32, StF64, false>(g, U, A, in, in_s, out, out_s, b, nrhs, s);
        default: break;
        }
    } else if (arith == QDD_PREC_DF64 && !b && op == QDD_PREC_F64) {
        QDD_TRY(ensure_copy(g, QDD_PREC_DF64, s));
        PrecCopy &c = g->copies[QDD_PREC_DF64];
        dim3 grid((g->hg.V + 127) / 128, nrhs);
        df kap = {(float)g->kappa, (float)(g->kappa - (double)(float)g->kappa)};
        LaunchScope ls(g->ctx->timer, K_DSLASH, s);
        const bool v256 = g->hg.Vd == 256;  // 4^4 domains: the volume fixed at compile time
        if (ip == QDD_PREC_F32 && v256)
            k_dslash_df<StF32, 256><<<grid, 128, 0, s>>>(g->geom, c.links.as<float4>(), c.clov.as<float4>(),
                                                         (const float2 *)in, (double2 *)out, kap);
        else if (ip == QDD_PREC_F32)
            k_dslash_df<StF32><<<grid, 128, 0, s>>>(g->geom, c.links.as<float4>(), c.clov.as<float4>(),
                                                    (const float2 *)in, (double2 *)out, kap);
        else if (ip == QDD_PREC_F64 && v256)
            k_dslash_df<StF64, 256><<<grid, 128, 0, s>>>(g->geom, c.links.as<float4>(), c.clov.as<float4>(),
                                                         (const double2 *)in, (double2 *)out, kap);
        else if (ip == QDD_PREC_F64)
            k_dslash_df<StF64><<<grid, 128, 0, s>>>(g->geom, c.links.as<float4>(), c.clov.as<float4>(),
                                                    (const double2 *)in, (double2 *)out, kap);
        else {
            set_error("double-float operator takes FP32 or FP64 input");
            return QDD_EINVAL;
        }
        QDD_CUDA(cudaGetLastError());
        return QDD_OK;
    } else if (arith == QDD_PREC_F32 && !b) {
        QDD_TRY(ensure_copy(g, fp, s));
        PrecCopy &c = g->copies[fp];
        switch (fp) {
        case QDD_PREC_F32: {
            Field<StF32> A{c.clov.as<float2>(), nullptr};
            if (ip == QDD_PREC_F32 && op == QDD_PREC_F32)
                return run_dslash_lowp<StF32, StF32, StF32, StF32>(g, fp, A, in, in_s, out, out_s, nrhs, s);
            if (ip == QDD_PREC_F32 && op == QDD_PREC_F64)
                return run_dslash_lowp<StF32, StF32, StF32, StF64>(g, fp, A, in, in_s, out, out_s, nrhs, s);
            break;
        }
        case QDD_PREC_F16S: {
            Field<StF16> A{c.clov.as<__half2>(), c.clov_s.as<float>()};
            if (ip == QDD_PREC_F16S && op == QDD_PREC_F16S)
                return run_dslash_lowp<StF16, StF16, StF16, StF16>(g, fp, A, in, in_s, out, out_s, nrhs, s);
            if (ip == QDD_PREC_F32 && op == QDD_PREC_F32)  // half links/clover, single spinors
                return run_dslash_lowp<StF16, StF16, StF32, StF32>(g, fp, A, in, in_s, out, out_s, nrhs, s);
            break;
        }
        case QDD_PREC_BF16S: {
            Field<StBF16> A{c.clov.as<__nv_bfloat162>(), c.clov_s.as<float>()};
            if (ip == QDD_PREC_BF16S && op == QDD_PREC_BF16S)
                return run_dslash_lowp<StBF16, StBF16, StBF16, StBF16>(g, fp, A, in, in_s, out, out_s, nrhs, s);
            break;
        }
        default: break;
        }
    }
    set_error("unsupported operator precision combination (arith %d, fields %d, in %d, out %d)", (int)arith, (int)fp,
              (int)ip, (int)op);
    return QDD_EINVAL;
}

}  // namespace qdd
