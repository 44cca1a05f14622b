// Shared device-side definitions of libqdd: complex arithmetic, storage
// precisions, the domain-blocked field layout and the spin algebra of the
// Wilson-clover operator (arXiv:1502.04025, Sec. 3.1-3.2).
//
// Device layout of every lattice field (Sec. 3.2 chooses a layout for the
// domain-decomposed algorithm; this one is chosen for coalesced GPU access
// and for one contiguous block per domain, so a domain stages with a single
// bulk copy):
//   domain slot d  : colour-major, d = colour*(Nd/2) + (block index >> 1)
//   site slot s    : parity-split within the domain, s = parity*(Vd/2) + (l >> 1),
//                    l the domain-local lexicographic index
//   element        : plane-major per domain, field[(d*planes + p)*Vd + s],
//                    one complex number per plane entry
// Planes: spinor 12 (p = spin*3 + colour); links 36 (p = mu*9 + a*3 + b);
// clover 36 (18 per chirality block: 3 pairs of real diagonal entries, then
// the 15 upper off-diagonal entries row by row).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace qdd {

// ------------------------------------------------------------------ complex

template <typename R>
struct cpx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a and -i * a
template <typename R>
__device__ __forceinline__ cpx<R> ti(cpx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cpx<R> tmi(cpx<R> a) { return {a.im, -a.re}; }
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(cpx<R> &acc, cpx<R> a, cpx<R> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cfmac(cpx<R> &acc, cpx<R> a, cpx<R> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// --------------------------------------------------------- storage formats

// One complex number per plane entry.  16-bit formats of spinors and clover
// carry one FP32 scale per site (stored value = value / scale); links are
// stored unscaled (unitary, |U_ab| <= 1).
struct StF64 {
    using T2 = double2;
    static constexpr bool kScaled = false;
    static constexpr int kBytes = 16;
    static constexpr bool kQuad = false;  // spinor fields in quad planes
};
struct StF32 {
    using T2 = float2;
    static constexpr bool kScaled = false;
    static constexpr int kBytes = 8;
    static constexpr bool kQuad = false;  // spinor fields in quad planes
};
struct StF16 {
    using T2 = __half2;
    static constexpr bool kScaled = true;
    static constexpr int kBytes = 4;
    static constexpr bool kQuad = true;  // spinor fields in quad planes
};
struct StBF16 {
    using T2 = __nv_bfloat162;
    static constexpr bool kScaled = true;
    static constexpr int kBytes = 4;
    static constexpr bool kQuad = false;  // spinor fields in quad planes
};

template <typename R>
__device__ __forceinline__ cpx<R> ld_c(const double2 *p) { double2 v = __ldg(p); return {(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> ld_c(const float2 *p) { float2 v = __ldg(p); return {(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> ld_c(const __half2 *p)
{
    float2 v = __half22float2(__ldg(p));
    return {(R)v.x, (R)v.y};
}
template <typename R>
__device__ __forceinline__ cpx<R> ld_c(const __nv_bfloat162 *p)
{
    float2 v = __bfloat1622float2(__ldg(p));
    return {(R)v.x, (R)v.y};
}

// plain (coherent) loads, for shared memory or buffers written in the same kernel
template <typename R>
__device__ __forceinline__ cpx<R> ld_s(const double2 *p) { double2 v = *p; return {(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> ld_s(const float2 *p) { float2 v = *p; return {(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> ld_s(const __half2 *p) { float2 v = __half22float2(*p); return {(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> ld_s(const __nv_bfloat162 *p)
{
    float2 v = __bfloat1622float2(*p);
    return {(R)v.x, (R)v.y};
}

template <typename R>
__device__ __forceinline__ void st_c(double2 *p, cpx<R> v) { *p = make_double2((double)v.re, (double)v.im); }
template <typename R>
__device__ __forceinline__ void st_c(float2 *p, cpx<R> v) { *p = make_float2((float)v.re, (float)v.im); }
template <typename R>
__device__ __forceinline__ void st_c(__half2 *p, cpx<R> v) { *p = __floats2half2_rn((float)v.re, (float)v.im); }
template <typename R>
__device__ __forceinline__ void st_c(__nv_bfloat162 *p, cpx<R> v)
{
    *p = __floats2bfloat162_rn((float)v.re, (float)v.im);
}

// A field in device memory: planes of Vd complex per domain, optional scale.
template <typename S>
struct Field {
    typename S::T2 *p;
    float *scale;  // [Nd*Vd], only for S::kScaled
};

// Spinor fields: per right-hand side and domain, a block of 12*Vd complex
// components.  Plane storage (FP64, FP32, BF16) keeps plane k of the block for
// component k of the domain's sites (offset k*Vd + s).  FP16 storage keeps
// quad planes: components 4q..4q+3 of a site side by side (16 bytes, one
// vector access), quad q of all the domain's sites before quad q+1 (offset
// (k/4)*4*Vd + 4s + k%4).  A 16-bit field's per-site scale is indexed by site.
// (Quad planes took the FP16 operator on 32^3x64 from 173.0 to 165.7 us; the
// BF16 operator measured 177.7 us in planes and 180.3 us in quads, so it keeps
// planes.)
__device__ __forceinline__ float2 word_f2(uint32_t w, const __half2 *)
{
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
}
__device__ __forceinline__ float2 word_f2(uint32_t w, const __nv_bfloat162 *)
{
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ uint32_t f2_word(float a, float b, const __half2 *)
{
    __half2 h = __floats2half2_rn(a, b);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
}
__device__ __forceinline__ uint32_t f2_word(float a, float b, const __nv_bfloat162 *)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
}

// The 12 stored components of site s of a spinor domain block blk (unscaled).
// NC: through the read-only path (the kernel does not write the field).
template <typename R, typename S, bool NC = true>
__device__ __forceinline__ void ld_sp_site(const typename S::T2 *blk, int s, int Vd, cpx<R> *x)
{
    if constexpr (S::kQuad) {
        const uint4 *q = reinterpret_cast<const uint4 *>(blk) + s;
        const typename S::T2 *tag = nullptr;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const uint4 w = NC ? __ldg(q + (int64_t)j * Vd) : q[(int64_t)j * Vd];
            const float2 a = word_f2(w.x, tag), b = word_f2(w.y, tag), c = word_f2(w.z, tag), e = word_f2(w.w, tag);
            x[4 * j + 0] = {(R)a.x, (R)a.y};
            x[4 * j + 1] = {(R)b.x, (R)b.y};
            x[4 * j + 2] = {(R)c.x, (R)c.y};
            x[4 * j + 3] = {(R)e.x, (R)e.y};
        }
    } else {
        const typename S::T2 *p = blk + s;
#pragma unroll
        for (int k = 0; k < 12; k++) x[k] = NC ? ld_c<R>(p + (int64_t)k * Vd) : ld_s<R>(p + (int64_t)k * Vd);
    }
}

// Store the 12 components x (already divided by the site's scale for 16-bit
// storage) of site s of a spinor domain block blk.
template <typename R, typename S>
__device__ __forceinline__ void st_sp_site(typename S::T2 *blk, int s, int Vd, const cpx<R> *x)
{
    if constexpr (S::kQuad) {
        uint4 *q = reinterpret_cast<uint4 *>(blk) + s;
        const typename S::T2 *tag = nullptr;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            uint4 w;
            w.x = f2_word((float)x[4 * j + 0].re, (float)x[4 * j + 0].im, tag);
            w.y = f2_word((float)x[4 * j + 1].re, (float)x[4 * j + 1].im, tag);
            w.z = f2_word((float)x[4 * j + 2].re, (float)x[4 * j + 2].im, tag);
            w.w = f2_word((float)x[4 * j + 3].re, (float)x[4 * j + 3].im, tag);
            q[(int64_t)j * Vd] = w;
        }
    } else {
        typename S::T2 *p = blk + s;
#pragma unroll
        for (int k = 0; k < 12; k++) st_c<R>(p + (int64_t)k * Vd, x[k]);
    }
}

// ------------------------------------------------------------------ geometry

// Direction k = 2*mu + b: b = 0 the forward neighbour n+mu, b = 1 the backward n-mu.
struct Geom {
    int L[4], dom[4], nb[4];
    int V, Vd, Vh, Nd, Nd2;
    int vd_shift;          // log2(Vd) when Vd is a power of two, else -1
    const uint16_t *nbl;   // [Vd][8]: neighbour site slot (wrapped into the domain), bit 15 = leaves the domain
    const int *nbd;        // [Nd][8]: neighbour domain slot
    const int *block_slot; // [Nd]: slot of the domain with lexicographic block index b
    // Face slots of a domain (one per hop that leaves it): direction dir's
    // slots start at foff[dir] and are indexed by the site's coordinates
    // transverse to mu = dir/2, which a hop and its reverse share.
    const uint32_t *fcoord;  // [Vd]: byte mu = transverse index of the site for direction mu
    int foff[8];
    int nf;                  // face slots per domain
};

// Site of thread index gi when the lattice is walked domain by domain in
// lexicographic block order (neighbouring domains close together in time, so
// their data is still in L2 when it is read as a neighbour); the storage
// order of the slots is colour-major.
__device__ __forceinline__ void lex_site(const Geom &g, int gi, int &d, int &s)
{
    int b;
    if (g.vd_shift >= 0) {
        b = gi >> g.vd_shift;
        s = gi & (g.Vd - 1);
    } else {
        b = gi / g.Vd;
        s = gi - b * g.Vd;
    }
    d = __ldg(g.block_slot + b);
}

constexpr uint16_t kCross = 0x8000;
constexpr uint16_t kSlotMask = 0x7fff;

__device__ __forceinline__ void split_index(const Geom &g, int gi, int &d, int &s)
{
    if (g.vd_shift >= 0) {
        d = gi >> g.vd_shift;
        s = gi & (g.Vd - 1);
    } else {
        d = gi / g.Vd;
        s = gi - d * g.Vd;
    }
}

// global index of the neighbour of (d, s) in direction k
__device__ __forceinline__ int neighbour(const Geom &g, int d, int s, int k)
{
    uint16_t e = __ldg(g.nbl + s * 8 + k);
    int nd = (e & kCross) ? __ldg(g.nbd + d * 8 + k) : d;
    return nd * g.Vd + (e & kSlotMask);
}

// plane-major address: global index gi = d*Vd + s, plane p of P
__device__ __forceinline__ int64_t paddr(const Geom &g, int gi, int p, int P)
{
    int d, s;
    split_index(g, gi, d, s);
    return ((int64_t)d * P + p) * g.Vd + s;
}

// ------------------------------------------------------------ spin algebra

// Spinor component index: spin*3 + colour.  In the chiral basis
//   gamma_mu = [[0, a_mu], [a_mu^+, 0]] (2x2 spin blocks),
//   a_x = -i sigma_x, a_y = -i sigma_y, a_z = -i sigma_z, a_t = 1.
// (1 - sgn*gamma_mu) psi = (h ; -sgn * a^+ h) with h = u - sgn * a l, where
// u = spins (0,1) and l = spins (2,3) of psi.  The hopping term only needs the
// two-spin vector h per colour (the rank-2 projection), so each hop costs two
// SU(3) products.

// h = u - sgn * (a_mu l): half spinor from a full spinor, per colour c
template <int MU, int SGN, typename R>
__device__ __forceinline__ void project(const cpx<R> *x, cpx<R> *h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> u0 = x[0 * 3 + c], u1 = x[1 * 3 + c], l0 = x[2 * 3 + c], l1 = x[3 * 3 + c];
        cpx<R> al0, al1;
        if (MU == 0) { al0 = tmi(l1); al1 = tmi(l0); }       // -i sigma_x l
        else if (MU == 1) { al0 = -l1; al1 = l0; }           // -i sigma_y l
        else if (MU == 2) { al0 = tmi(l0); al1 = ti(l1); }   // -i sigma_z l
        else { al0 = l0; al1 = l1; }                         // 1 l
        if (SGN > 0) { h[c] = u0 - al0; h[3 + c] = u1 - al1; }
        else { h[c] = u0 + al0; h[3 + c] = u1 + al1; }
    }
}

// acc += (w ; -sgn * a_mu^+ w), w the half spinor after the colour product.
// SWAP: acc holds spins (2,3) in its first six entries and spins (0,1) in
// its last six (the same sums, stored the other way round).
template <int MU, int SGN, bool SWAP = false, typename R>
__device__ __forceinline__ void reconstruct_add(const cpx<R> *w, cpx<R> *acc)
{
    constexpr int up = SWAP ? 6 : 0, lo = SWAP ? 0 : 6;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> w0 = w[c], w1 = w[3 + c];
        cpx<R> b0, b1;  // a^+ w
        if (MU == 0) { b0 = ti(w1); b1 = ti(w0); }          // i sigma_x w
        else if (MU == 1) { b0 = w1; b1 = -w0; }            // i sigma_y w
        else if (MU == 2) { b0 = ti(w0); b1 = tmi(w1); }    // i sigma_z w
        else { b0 = w0; b1 = w1; }
        acc[up + c] = acc[up + c] + w0;
        acc[up + 3 + c] = acc[up + 3 + c] + w1;
        if (SGN > 0) { acc[lo + c] = acc[lo + c] - b0; acc[lo + 3 + c] = acc[lo + 3 + c] - b1; }
        else { acc[lo + c] = acc[lo + c] + b0; acc[lo + 3 + c] = acc[lo + 3 + c] + b1; }
    }
}

// FP32 form of su3_mul_half: the two spins of h share every link entry, so
// their products run as pairs (one paired FMA for the two spins), with the
// scalar form's order of operations in each lane -- the same bits.
template <bool DAG>
__device__ __forceinline__ void su3_mul_half_x2(const cpx<float> *U, const cpx<float> *h, cpx<float> *w)
{
    float2 hr[3], hi[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        hr[b] = make_float2(h[b].re, h[3 + b].re);
        hi[b] = make_float2(h[b].im, h[3 + b].im);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const cpx<float> u = DAG ? U[b * 3 + a] : U[a * 3 + b];
            const float2 ur = make_float2(u.re, u.re);
            const float2 ui = make_float2(DAG ? u.im : -u.im, DAG ? u.im : -u.im);  // enters re
            const float2 uj = make_float2(DAG ? -u.im : u.im, DAG ? -u.im : u.im);  // enters im
            ar = __ffma2_rn(ur, hr[b], ar);
            ar = __ffma2_rn(ui, hi[b], ar);
            ai = __ffma2_rn(ur, hi[b], ai);
            ai = __ffma2_rn(uj, hr[b], ai);
        }
        w[a] = mk(ar.x, ai.x);
        w[3 + a] = mk(ar.y, ai.y);
    }
}

// w = U h (DAG = false) or U^+ h (DAG = true) for the two spins of h;
// PAIRED: the FP32 form runs the two spins as paired FMAs (same bits)
template <bool DAG, typename R, bool PAIRED = true>
__device__ __forceinline__ void su3_mul_half(const cpx<R> *U, const cpx<R> *h, cpx<R> *w)
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (sizeof(R) == 4 && PAIRED) {
        su3_mul_half_x2<DAG>(U, h, w);
        return;
    }
#endif
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cpx<R> acc = mk<R>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (DAG) cfmac(acc, U[b * 3 + a], h[sp * 3 + b]);
                else cfma(acc, U[a * 3 + b], h[sp * 3 + b]);
            }
            w[sp * 3 + a] = acc;
        }
}

// one hop: acc += (1 - sgn gamma_mu) V x, V = U (forward) or U^+ (backward)
// reconstruct_add with a weight m (1: the same sums, as single-rounded
// fused multiply-adds of 1 * w; 0: acc unchanged), for hops that every lane
// evaluates and only some keep
template <int MU, int SGN, typename R>
__device__ __forceinline__ void reconstruct_fma(R m, const cpx<R> *w, cpx<R> *acc)
{
    const R ms = SGN > 0 ? -m : m;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> w0 = w[c], w1 = w[3 + c];
        cpx<R> b0, b1;  // a^+ w
        if (MU == 0) { b0 = ti(w1); b1 = ti(w0); }
        else if (MU == 1) { b0 = w1; b1 = -w0; }
        else if (MU == 2) { b0 = ti(w0); b1 = tmi(w1); }
        else { b0 = w0; b1 = w1; }
        acc[c] = mk<R>(fma(m, w0.re, acc[c].re), fma(m, w0.im, acc[c].im));
        acc[3 + c] = mk<R>(fma(m, w1.re, acc[3 + c].re), fma(m, w1.im, acc[3 + c].im));
        acc[6 + c] = mk<R>(fma(ms, b0.re, acc[6 + c].re), fma(ms, b0.im, acc[6 + c].im));
        acc[9 + c] = mk<R>(fma(ms, b1.re, acc[9 + c].re), fma(ms, b1.im, acc[9 + c].im));
    }
}

template <int MU, int SGN, bool SWAP = false, typename R>
__device__ __forceinline__ void hop(const cpx<R> *U, const cpx<R> *x, cpx<R> *acc)
{
    cpx<R> h[6], w[6];
    project<MU, SGN>(x, h);
    su3_mul_half<(SGN < 0)>(U, h, w);
    reconstruct_add<MU, SGN, SWAP>(w, acc);
}

// Hermitian 6x6 block from its packed 18 complex slots
template <typename R>
__device__ __forceinline__ void herm6_mul(const cpx<R> *blk, const cpx<R> *in, cpx<R> *out)
{
    R d[6] = {blk[0].re, blk[0].im, blk[1].re, blk[1].im, blk[2].re, blk[2].im};
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = d[i] * in[i];
    int k = 3;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            cfma(out[i], blk[k], in[j]);
            cfmac(out[j], blk[k], in[i]);
            k++;
        }
}

// FP32 form of the two clover blocks at once: block 0 (spins 0,1) in lane 0
// and block 1 (spins 2,3) in lane 1 of paired FMAs.  Each lane runs
// herm6_mul's sequence of operations, so the result is the same bits.
__device__ __forceinline__ void herm6_mul_x2(const cpx<float> *b0, const cpx<float> *b1, const cpx<float> *in,
                                             cpx<float> *out)
{
    float2 inr[6], ini[6], ore[6], oim[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        inr[i] = make_float2(in[i].re, in[6 + i].re);
        ini[i] = make_float2(in[i].im, in[6 + i].im);
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const float2 dd = make_float2((i & 1) ? b0[i >> 1].im : b0[i >> 1].re, (i & 1) ? b1[i >> 1].im : b1[i >> 1].re);
        ore[i] = __fmul2_rn(dd, inr[i]);
        oim[i] = __fmul2_rn(dd, ini[i]);
    }
    int k = 3;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const float2 br = make_float2(b0[k].re, b1[k].re), bi = make_float2(b0[k].im, b1[k].im);
            const float2 nbi = make_float2(-b0[k].im, -b1[k].im);
            ore[i] = __ffma2_rn(br, inr[j], ore[i]);  // out[i] += b in[j]
            ore[i] = __ffma2_rn(nbi, ini[j], ore[i]);
            oim[i] = __ffma2_rn(br, ini[j], oim[i]);
            oim[i] = __ffma2_rn(bi, inr[j], oim[i]);
            ore[j] = __ffma2_rn(br, inr[i], ore[j]);  // out[j] += conj(b) in[i]
            ore[j] = __ffma2_rn(bi, ini[i], ore[j]);
            oim[j] = __ffma2_rn(br, ini[i], oim[j]);
            oim[j] = __ffma2_rn(nbi, inr[i], oim[j]);
            k++;
        }
#pragma unroll
    for (int i = 0; i < 6; i++) {
        out[i] = mk(ore[i].x, oim[i].x);
        out[6 + i] = mk(ore[i].y, oim[i].y);
    }
}

// ------------------------------------------------------------ double-float
//
// A value hi + lo held in two FP32 numbers (|lo| <= ulp(hi)/2), for operator
// applications that need FP64-class accuracy on a GPU whose FP64 pipe is far
// slower than its FP32 pipe.  Built from error-free transformations (Knuth's
// TwoSum, Dekker's FastTwoSum, and the FMA form of the exact product); the
// intrinsics keep the compiler from contracting or reordering them.

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b for double-floats
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = df_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// compensated accumulator: s collects the leading parts with TwoSum, c the
// rounding errors and low-order terms; value = s + c
struct dfacc {
    float s, c;
};

__device__ __forceinline__ void dfacc_zero(dfacc &a) { a.s = 0.f; a.c = 0.f; }

// acc += x * y (x, y double-floats; the lo*lo term, below 2^-46 relative, is dropped)
__device__ __forceinline__ void dfacc_mul_add(dfacc &acc, df x, df y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    df t = df_two_sum(acc.s, p);
    acc.s = t.hi;
    acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, e));
}

// acc += x
__device__ __forceinline__ void dfacc_add(dfacc &acc, df x)
{
    df t = df_two_sum(acc.s, x.hi);
    acc.s = t.hi;
    acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ df dfacc_value(const dfacc &a) { return df_fast_two_sum(a.s, a.c); }

__device__ __forceinline__ df df_from_double(double v)
{
    float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// complex double-float
struct cdf {
    df re, im;
};

__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
__device__ __forceinline__ cdf cdf_ti(cdf a) { return {df_neg(a.im), a.re}; }   // i * a
__device__ __forceinline__ cdf cdf_tmi(cdf a) { return {a.im, df_neg(a.re)}; }  // -i * a
__device__ __forceinline__ cdf cdf_neg(cdf a) { return {df_neg(a.re), df_neg(a.im)}; }

struct cdfacc {
    dfacc re, im;
};

__device__ __forceinline__ void cdfacc_zero(cdfacc &a) { dfacc_zero(a.re); dfacc_zero(a.im); }

// acc += a * b (CONJ: conj(a) * b)
template <bool CONJ>
__device__ __forceinline__ void cdfacc_mul_add(cdfacc &acc, cdf a, cdf b)
{
    dfacc_mul_add(acc.re, a.re, b.re);
    dfacc_mul_add(acc.re, CONJ ? a.im : df_neg(a.im), b.im);
    dfacc_mul_add(acc.im, a.re, b.im);
    dfacc_mul_add(acc.im, CONJ ? df_neg(a.im) : a.im, b.re);
}

__device__ __forceinline__ cdf cdfacc_value(const cdfacc &a) { return {dfacc_value(a.re), dfacc_value(a.im)}; }

// Storage of a double-float complex number: (re.hi, re.lo, im.hi, im.lo).
struct StDF {
    using T2 = float4;
    static constexpr bool kScaled = false;
    static constexpr int kBytes = 16;
};

// Runtime-checked device error flags (bounded waits that ran out, etc.).
constexpr int kErrMbarTimeout = 1;

// Range checks of the hot-path kernels' indices.  A library built with
// -DQDD_CHECK tests every guarded index; one out of range is counted in this
// translation unit's counter and its access skipped (no trap, no wait).  In
// the normal build the guard is the constant true and compiles away.
#ifdef QDD_CHECK
static __device__ unsigned long long g_check_hits;
__device__ __forceinline__ bool in_range(long long v, long long lo, long long hi)
{
    if (v >= lo && v < hi) return true;
    atomicAdd(&g_check_hits, 1ull);
    return false;
}
#define QDD_IN_RANGE(v, lo, hi) ::qdd::in_range((long long)(v), (long long)(lo), (long long)(hi))
#else
#define QDD_IN_RANGE(v, lo, hi) true
#endif

}  // namespace qdd
