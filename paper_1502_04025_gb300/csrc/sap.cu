// Schwarz alternating procedure (multiplicative Schwarz), one colour half-sweep
// per launch (arXiv:1502.04025, Sec. 3.1; Sec. 3.5: cores synchronise only
// after an MR block solve, here the kernel boundary).
//
// One CTA per domain Lambda of the colour being swept, one thread per
// even/odd site pair (k_sap), or two threads per site pair, each with two of
// the four directions and one clover block (k_sap_pair, the form for FP32
// links; see there).  The domain's links and Schwarz clover blocks (A on even
// sites, A^{-1} on odd sites) are staged into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier) when they fit; Sec. 3.3
// keeps each domain resident in a core's L2 for the same reason.  Then:
//
//   rho_Lambda += kappa * (hops into Lambda from the other colour's last
//                  corrections, read from Lambda's face slots)
//   bhat_e = rho_e - D_eo A_oo^{-1} rho_o           (even-odd Schur RHS)
//   x_e = 0, r = bhat_e; nmr times:                  (MR on Dhat, Sec. 3.1 footnote)
//       p = Dhat r = A_ee r - D_eo A_oo^{-1} D_oe r   (hops leaving Lambda dropped)
//       alpha = <p, r> / <p, p>;  x_e += alpha r;  r -= alpha p
//   x_o = A_oo^{-1}(rho_o - D_oe x_e)
//   delta = (x_e, x_o);  psi_Lambda += delta;  rho_Lambda = (r, 0)
//   the hops of delta out of Lambda -> the neighbours' face slots
//
// D_eo = -kappa H_eo, D_oe = -kappa H_oe.  The odd half of the new domain
// residual is zero and the even half is the MR residual, so the residual on
// Lambda is set directly.  The neighbours receive -D delta (the inter-domain
// update, Sec. 3.2) at the start of the next half-sweep: each hop of delta
// out of Lambda, projected and multiplied by its link while delta is still in
// registers, goes to the face slot of the receiving site and direction.  Every
// slot has one writer, and the receiving site sums its slots in a fixed
// direction order, so there are no atomics and results are deterministic.
// Domain dot products: warp shuffles, then a fixed-order sum over warps in
// shared memory (deterministic).
#include <type_traits>

#include "internal.h"

namespace qdd {

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false if the barrier did not complete within max_spins polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t max_spins)
{
    for (uint32_t n = 0; n < max_spins; n++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Programmatic dependent launch: let the next half-sweep's CTAs start (they
// stage their read-only domain data), and wait for the previous grid's
// results before reading them.  Both are no-ops without a dependent launch.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// order this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a CTA barrier) before later bulk async copies into them
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// pull bytes (multiple of 16, 16-aligned) into L2 ahead of use; no completion
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes)
{
    const uint32_t kChunk = 32768;
    for (uint32_t off = 0; off < bytes; off += kChunk) {
        uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char *)src + off), "r"(n) : "memory");
    }
}

// copy bytes (multiple of 16, both addresses 16-aligned) in chunks
__device__ __forceinline__ void bulk_g2s_chunked(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    const uint32_t kChunk = 32768;
    for (uint32_t off = 0; off < bytes; off += kChunk) {
        uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
        bulk_g2s((char *)dst + off, (const char *)src + off, n, bar);
    }
}

// Poll limit of the first bounded wait of a visit (the staging of links and
// clover).  The range-checked build lets a test lower it, so that the wait
// gives up and the timeout path runs: the kernel flags the error, lets its
// copies land within the drain wait's own limit and leaves.
#ifdef QDD_CHECK
static __device__ unsigned g_first_wait_spins = 1u << 22;
#define QDD_FIRST_WAIT_SPINS g_first_wait_spins
#else
#define QDD_FIRST_WAIT_SPINS (1u << 22)
#endif

// ---------------------------------------------------------- kernel state

template <typename R, typename SL, typename SC, typename SS, typename SP>
struct SapArgs {
    Geom g;
    Field<SL> U;
    Field<SC> C;      // Schwarz clover: A on even sites, A^{-1} on odd sites
    Field<SS> rho;    // residual (read and written on the swept domains)
    cpx<R> *face;     // face slots: [rhs][domain][6][nf] projected hops into each domain
    Field<SP> psi;    // accumulated preconditioner output
    int64_t rstride;  // elements between right-hand sides (V*12)
    int64_t sstride;  // scale entries between right-hand sides (V)
    int64_t fstride;  // face elements between right-hand sides (Nd*6*nf)
    R kappa;
    int colour, nmr, nrhs, first_psi, gather;
    int *err;
    // the domains of this launch: block b sweeps domain colour*Nd/2 + dfirst +
    // (b < nsplit ? b : b + dskip); one launch over all of a colour's
    // domains is (0, grid, 0); a sharded field sweeps its boundary t-blocks
    // first and its interior second
    int dfirst, nsplit, dskip, nblocks;  // nblocks: the grid
};

// block b's domain in a launch
template <typename A>
__device__ __forceinline__ int sap_domain(const A &a, int Nd2, int b)
{
    return a.colour * Nd2 + a.dfirst + (b < a.nsplit ? b : b + a.dskip);
}


__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

// entries of the MR reduction buffer: 4 per warp when the half-field fills
// whole warps, else one triple per thread (3 * Vh)
__host__ __device__ constexpr int sap_red_elems(int Vh) { return (Vh % 32 == 0 || 3 * Vh <= 128) ? 128 : 3 * Vh; }

template <typename R, typename SL, typename SC>
__host__ __device__ constexpr size_t sap_smem_layout(int Vd, bool stl, bool stc)
{
    return (stl ? align128((size_t)36 * Vd * sizeof(typename SL::T2)) : 0) +
           (stc ? align128((size_t)36 * Vd * sizeof(typename SC::T2)) : 0) +
           ((stc && SC::kScaled) ? align128((size_t)Vd * 4) : 0) + 3 * align128((size_t)12 * (Vd / 2) * sizeof(cpx<R>)) +
           align128((size_t)sap_red_elems(Vd / 2) * sizeof(R)) + align128(16);
}

// Shared-memory half-fields: 12 components of Vh sites.  PP (FP32 only): pair
// planes, components 2q and 2q+1 of a site side by side, so that one 16-byte
// access moves two (element (q*Vh + s)*2 + k%2 for k = 2q, 2q+1); else planes
// (element k*Vh + s).  hf_load/hf_store move N components from k0 (even).
// The paired-thread form uses pair planes (32^3x64 FP32: 0.682 -> 0.651 ms
// per half-sweep); the one-thread form measured slower with them (48^3x96
// BF16: 2.300 -> 2.343 ms) and keeps planes.
template <int N, bool PP, typename R>
__device__ __forceinline__ void hf_load(const cpx<R> *f, int k0, int s, int Vh, cpx<R> *x)
{
    if constexpr (PP && sizeof(R) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(f);
#pragma unroll
        for (int j = 0; j < N / 2; j++) {
            const float4 w = q[((k0 >> 1) + j) * Vh + s];
            x[2 * j] = {w.x, w.y};
            x[2 * j + 1] = {w.z, w.w};
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; k++) x[k] = f[(k0 + k) * Vh + s];
    }
}

template <int N, bool PP, typename R>
__device__ __forceinline__ void hf_store(cpx<R> *f, int k0, int s, int Vh, const cpx<R> *x)
{
    if constexpr (PP && sizeof(R) == 4) {
        float4 *q = reinterpret_cast<float4 *>(f);
#pragma unroll
        for (int j = 0; j < N / 2; j++)
            q[((k0 >> 1) + j) * Vh + s] = make_float4(x[2 * j].re, x[2 * j].im, x[2 * j + 1].re, x[2 * j + 1].im);
    } else {
#pragma unroll
        for (int k = 0; k < N; k++) f[(k0 + k) * Vh + s] = x[k];
    }
}

// One-thread form: the hops in x, y and z without divergent branches (see
// inner_dir_e): every lane has some neighbours inside the domain and some
// outside, so the warp runs each hop body anyway, and without the branches
// the compiler schedules across hops (48^3x96 BF16: 2.298 -> 2.283 ms per
// half-sweep, the same bits).  The t hops keep their branches: a warp of
// sites on a t face of the domain skips one of them whole (branch-free t
// measured 2.316 ms).  With 16-bit links only: the one-thread form with FP32
// links (8x4^3 domains, 16^3x32) measured slower branch-free (50.1 against
// 48.9 us per half-sweep).
constexpr bool kBranchFreeHops = true;

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC, bool PP = false>
struct SapBlock {
    const SapArgs<R, SL, SC, SS, SP> &a;
    const Geom &g;  // the kernel's geometry (with compile-time fields for a fixed domain shape)
    int d, Vd, Vh;
    const typename SL::T2 *sL;
    const typename SC::T2 *sC;
    const float *sCs;

    __device__ __forceinline__ void link(int dd, int s, int mu, cpx<R> *u) const
    {
        if (STL && dd == d) {
#pragma unroll
            for (int k = 0; k < 9; k++) u[k] = ld_s<R>(sL + (mu * 9 + k) * Vd + s);
        } else {
            const typename SL::T2 *p = a.U.p + ((int64_t)dd * 36 + mu * 9) * Vd + s;
#pragma unroll
            for (int k = 0; k < 9; k++) u[k] = ld_c<R>(p + (int64_t)k * Vd);
        }
    }

    // out = C(s) in : the Schwarz clover of this domain's site s, both blocks;
    // a 16-bit clover's per-site scale multiplies the 12 products, not the 36
    // stored entries
    __device__ __forceinline__ void clover(int s, const cpx<R> *in, cpx<R> *out) const
    {
        cpx<R> m[2][18];
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            if (STC) {
#pragma unroll
                for (int k = 0; k < 18; k++) m[blk][k] = ld_s<R>(sC + (blk * 18 + k) * Vd + s);
            } else {
                const typename SC::T2 *p = a.C.p + ((int64_t)d * 36 + blk * 18) * Vd + s;
#pragma unroll
                for (int k = 0; k < 18; k++) m[blk][k] = ld_c<R>(p + (int64_t)k * Vd);
            }
        }
        if constexpr (sizeof(R) == 4) {
            herm6_mul_x2(m[0], m[1], in, out);  // both blocks in paired FMAs
        } else {
            herm6_mul(m[0], in, out);
            herm6_mul(m[1], in + 6, out + 6);
        }
        if (SC::kScaled) {
            const R sc = STC ? (R)sCs[s] : (R)__ldg(a.C.scale + (int64_t)d * Vd + s);
#pragma unroll
            for (int k = 0; k < 12; k++) out[k] = sc * out[k];
        }
    }

    // out = block b (0: spins 0,1; 1: spins 2,3) of C(s) applied to the six
    // components in (the paired-thread form's share of the clover)
    __device__ __forceinline__ void clover_blk(int s, int b, const cpx<R> *in, cpx<R> *out) const
    {
        static_assert(STC, "the paired-thread form stages the clover");
        cpx<R> m[18];
#pragma unroll
        for (int k = 0; k < 18; k++) m[k] = ld_s<R>(sC + (b * 18 + k) * Vd + s);
        herm6_mul(m, in, out);
        if (SC::kScaled) {
            const R sc = (R)sCs[s];
#pragma unroll
            for (int k = 0; k < 6; k++) out[k] = sc * out[k];
        }
    }

    // hops of site s from a shared-memory half-field (sites src_off..src_off+Vh-1),
    // dropping hops that leave the domain (Dirichlet boundary); ef, eb: the
    // site's forward and backward neighbour entries in direction MU
    template <int MU, bool SWAP = false>
    __device__ __forceinline__ void inner_dir_e(int s, uint16_t ef, uint16_t eb, const cpx<R> *src, int src_off,
                                                cpx<R> *acc) const
    {
        if constexpr (kBranchFreeHops && !PP && !SWAP && sizeof(R) == 4 && MU < 3 && !std::is_same<SL, StF32>::value) {
            // every lane evaluates both hops (a dropped one from slot 0 with
            // its own link) and adds them with weight 1 or 0
            const bool okf = !(ef & kCross) && QDD_IN_RANGE((ef & kSlotMask) - src_off, 0, Vh);
            const bool okb = !(eb & kCross) && QDD_IN_RANGE((eb & kSlotMask) - src_off, 0, Vh);
            const int nf = okf ? (ef & kSlotMask) - src_off : 0;
            const int nbh = okb ? (eb & kSlotMask) - src_off : 0;
            const int nbs = okb ? (eb & kSlotMask) : s;
            cpx<R> u[9], x[12], h[6], w[6];
#pragma unroll
            for (int k = 0; k < 12; k++) x[k] = src[k * Vh + nf];
            link(d, s, MU, u);
            project<MU, +1>(x, h);
            su3_mul_half<false>(u, h, w);
            reconstruct_fma<MU, +1>(okf ? (R)1 : (R)0, w, acc);
#pragma unroll
            for (int k = 0; k < 12; k++) x[k] = src[k * Vh + nbh];
            link(d, nbs, MU, u);
            project<MU, -1>(x, h);
            su3_mul_half<true>(u, h, w);
            reconstruct_fma<MU, -1>(okb ? (R)1 : (R)0, w, acc);
            return;
        }
        cpx<R> u[9], x[12];
        if (!(ef & kCross) && QDD_IN_RANGE((ef & kSlotMask) - src_off, 0, Vh)) {
            int ns = (ef & kSlotMask) - src_off;
            if constexpr (PP) {
                hf_load<12, PP>(src, 0, ns, Vh, x);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) x[k] = src[k * Vh + ns];
            }
            link(d, s, MU, u);
            hop<MU, +1, SWAP>(u, x, acc);
        }
        if (!(eb & kCross) && QDD_IN_RANGE((eb & kSlotMask) - src_off, 0, Vh)) {
            int ns = eb & kSlotMask;
            if constexpr (PP) {
                hf_load<12, PP>(src, 0, ns - src_off, Vh, x);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) x[k] = src[k * Vh + ns - src_off];
            }
            link(d, ns, MU, u);
            hop<MU, -1, SWAP>(u, x, acc);
        }
    }

    template <int MU>
    __device__ __forceinline__ void inner_dir(int s, const uint16_t *nb, const cpx<R> *src, int src_off,
                                              cpx<R> *acc) const
    {
        inner_dir_e<MU>(s, nb[2 * MU], nb[2 * MU + 1], src, src_off, acc);
    }

    // Push the correction dl of site s across the domain faces, into the face
    // slot of the receiving site m and direction.  A site crossing +mu is m's
    // backward neighbour: the slot gets U_mu(s)^+ (1 + gamma_mu) dl projected
    // (this domain's link).  A site crossing -mu is m's forward neighbour: the
    // slot gets (1 - gamma_mu) dl projected, and m applies its own U_mu(m).
    // Either way each side reads only links it holds in shared memory.
    // fc: the site's packed transverse indices; nbd: this domain's neighbours
    template <int MU>
    __device__ __forceinline__ void face_out_dir(int s, const uint16_t *nb, uint32_t fc, const int *nbd,
                                                 const cpx<R> *dl, cpx<R> *fb) const
    {
        const int nf = g.nf, t = (fc >> (8 * MU)) & 255;
        cpx<R> h[6];
        if ((nb[2 * MU] & kCross) && QDD_IN_RANGE(nbd[2 * MU], 0, g.Nd) &&
            QDD_IN_RANGE(g.foff[2 * MU + 1] + t, 0, nf)) {
            cpx<R> u[9], w[6];
            project<MU, -1>(dl, h);
            link(d, s, MU, u);
            su3_mul_half<true>(u, h, w);
            cpx<R> *dst = fb + (int64_t)nbd[2 * MU] * 6 * nf + g.foff[2 * MU + 1] + t;
#pragma unroll
            for (int k = 0; k < 6; k++) dst[k * nf] = w[k];
        }
        if ((nb[2 * MU + 1] & kCross) && QDD_IN_RANGE(nbd[2 * MU + 1], 0, g.Nd) &&
            QDD_IN_RANGE(g.foff[2 * MU] + t, 0, nf)) {
            project<MU, +1>(dl, h);
            cpx<R> *dst = fb + (int64_t)nbd[2 * MU + 1] * 6 * nf + g.foff[2 * MU] + t;
#pragma unroll
            for (int k = 0; k < 6; k++) dst[k * nf] = h[k];
        }
    }

    __device__ __forceinline__ void face_out(int s, const uint16_t *nb, uint32_t fc, const int *nbd,
                                             const cpx<R> *dl, cpx<R> *fb) const
    {
        face_out_dir<0>(s, nb, fc, nbd, dl, fb);
        face_out_dir<1>(s, nb, fc, nbd, dl, fb);
        face_out_dir<2>(s, nb, fc, nbd, dl, fb);
        face_out_dir<3>(s, nb, fc, nbd, dl, fb);
    }

    __device__ __forceinline__ void inner_hops(int s, const uint16_t *nb, const cpx<R> *src, int src_off,
                                               cpx<R> *acc) const
    {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
        inner_dir<0>(s, nb, src, src_off, acc);
        inner_dir<1>(s, nb, src, src_off, acc);
        inner_dir<2>(s, nb, src, src_off, acc);
        inner_dir<3>(s, nb, src, src_off, acc);
    }

};

// acc = the hops into site s across its domain's faces, from the face slots
// fd of its domain (pushed by the neighbouring domains' last half-sweep; in
// shared or global memory), reconstructed to full spinors and summed in
// direction order.  A forward hop's slot holds the projected neighbour and
// needs this site's link U_mu(s), given by lnk(mu, u).
template <int MU, typename R, typename LinkFn>
__device__ __forceinline__ void face_in_dir(const Geom &g, const uint16_t *nb, uint32_t fc, const cpx<R> *fd,
                                            const LinkFn &lnk, cpx<R> *acc)
{
    const int t = (fc >> (8 * MU)) & 255;
    cpx<R> h[6];
    if ((nb[2 * MU] & kCross) && QDD_IN_RANGE(g.foff[2 * MU] + t, 0, g.nf)) {
        const cpx<R> *src = fd + g.foff[2 * MU] + t;
#pragma unroll
        for (int k = 0; k < 6; k++) h[k] = src[k * g.nf];
        cpx<R> u[9], w[6];
        lnk(MU, u);
        su3_mul_half<false>(u, h, w);
        reconstruct_add<MU, +1>(w, acc);
    }
    if ((nb[2 * MU + 1] & kCross) && QDD_IN_RANGE(g.foff[2 * MU + 1] + t, 0, g.nf)) {
        const cpx<R> *src = fd + g.foff[2 * MU + 1] + t;
#pragma unroll
        for (int k = 0; k < 6; k++) h[k] = src[k * g.nf];
        reconstruct_add<MU, -1>(h, acc);
    }
}

template <typename R, typename LinkFn>
__device__ __forceinline__ void face_in(const Geom &g, const uint16_t *nb, uint32_t fc, const cpx<R> *fd,
                                        const LinkFn &lnk, cpx<R> *acc)
{
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
    face_in_dir<0>(g, nb, fc, fd, lnk, acc);
    face_in_dir<1>(g, nb, fc, fd, lnk, acc);
    face_in_dir<2>(g, nb, fc, fd, lnk, acc);
    face_in_dir<3>(g, nb, fc, fd, lnk, acc);
}

template <typename R, typename S>
__device__ __forceinline__ void load_sp(const Field<S> &f, int64_t rb, int64_t sb, int d, int s, int Vd, cpx<R> *x)
{
    if constexpr (S::kQuad) {
        R sc = (R)f.scale[sb + (int64_t)d * Vd + s];
        ld_sp_site<R, S, false>(f.p + rb + (int64_t)d * 12 * Vd, s, Vd, x);
#pragma unroll
        for (int k = 0; k < 12; k++) x[k] = sc * x[k];
    } else {
        const typename S::T2 *p = f.p + rb + (int64_t)d * 12 * Vd + s;
        R sc = S::kScaled ? (R)f.scale[sb + (int64_t)d * Vd + s] : (R)1;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            cpx<R> v = ld_s<R>(p + (int64_t)k * Vd);
            x[k] = S::kScaled ? sc * v : v;
        }
    }
}

template <typename R, typename S>
__device__ __forceinline__ void store_sp(const Field<S> &f, int64_t rb, int64_t sb, int d, int s, int Vd,
                                         const cpx<R> *x)
{
    typename S::T2 *p = f.p + rb + (int64_t)d * 12 * Vd + s;
    if (S::kScaled) {
        R m = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) m = fmax(m, fmax(fabs(x[k].re), fabs(x[k].im)));
        float sc = (float)m;
        f.scale[sb + (int64_t)d * Vd + s] = sc;
        R inv = m > 0 ? (R)1 / (R)sc : (R)0;
        if constexpr (S::kQuad) {
            cpx<R> y[12];
#pragma unroll
            for (int k = 0; k < 12; k++) y[k] = inv * x[k];
            st_sp_site<R, S>(f.p + rb + (int64_t)d * 12 * Vd, s, Vd, y);
        } else {
#pragma unroll
            for (int k = 0; k < 12; k++) st_c<R>(p + (int64_t)k * Vd, inv * x[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 12; k++) st_c<R>(p + (int64_t)k * Vd, x[k]);
    }
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Phases of one domain visit.  Every phase runs the same code: one hop sum
// over the sites of one parity (read from the other parity's shared-memory
// half-field), one clover product, a short epilogue; the stencil and clover
// code therefore appear once in the kernel, which keeps it inside the
// instruction cache.
enum SapPhase : int {
    PH_SETUP_ODD = 0,   // t_o = A_oo^{-1} rho_o                      -> sT
    PH_SETUP_EVEN = 1,  // r = rho_e + kappa H_eo t_o ; x = 0           -> sR
    PH_MR_ODD = 2,      // t_o = A_oo^{-1} (-kappa H_oe r)              -> sT
    PH_MR_EVEN = 3,     // p = A_ee r + kappa H_eo t_o; MR update       -> sR
    PH_RECON_ODD = 4    // x_o = A_oo^{-1} (rho_o + kappa H_oe x_e)
};

// MAXT / MINB: the launch bounds.  The default form allows 256 threads (an
// 8x4^3 domain); the occupancy form (128 threads, 3 CTAs per SM) caps the
// registers at 170 so that three 4^4 domains run on an SM at once.
// The geometry of a domain shape fixed at compile time (SHAPE 1: 4^4,
// 2: 8x4^3; 0: taken from the arguments): the volume and the face-slot
// offsets become immediates in the stencil and the face code.
template <int SHAPE>
__device__ __forceinline__ Geom sap_geom(const Geom &g0)
{
    Geom g = g0;
    if (SHAPE > 0) {
        constexpr int dx = SHAPE == 1 ? 4 : 8, vd = dx * 64;
        constexpr int fx = vd / dx, fo = vd / 4;  // slots of an x face; of a y, z or t face
        g.Vd = vd;
        g.Vh = vd / 2;
        g.vd_shift = SHAPE == 1 ? 8 : 9;
        g.nf = 2 * (fx + 3 * fo);
        g.foff[0] = 0;
        g.foff[1] = fx;
        g.foff[2] = 2 * fx;
        g.foff[3] = 2 * fx + fo;
        g.foff[4] = 2 * fx + 2 * fo;
        g.foff[5] = 2 * fx + 3 * fo;
        g.foff[6] = 2 * fx + 4 * fo;
        g.foff[7] = 2 * fx + 5 * fo;
    }
    return g;
}

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC, int MAXT = 256,
          int MINB = 1, int SHAPE = 0>
__global__ void __launch_bounds__(MAXT, MINB) k_sap(const SapArgs<R, SL, SC, SS, SP> a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const Geom g = sap_geom<SHAPE>(a.g);
    const int Vd = g.Vd, Vh = g.Vh;
    const int i = threadIdx.x;
    const int bx = blockIdx.x;
    const int d = sap_domain(a, g.Nd2, bx);
    const int se = i, so = Vh + i;

    unsigned char *ptr = smem;
    typename SL::T2 *sL = nullptr;
    typename SC::T2 *sC = nullptr;
    float *sCs = nullptr;
    if (STL) { sL = (typename SL::T2 *)ptr; ptr += align128((size_t)36 * Vd * sizeof(typename SL::T2)); }
    if (STC) {
        sC = (typename SC::T2 *)ptr;
        ptr += align128((size_t)36 * Vd * sizeof(typename SC::T2));
        if (SC::kScaled) { sCs = (float *)ptr; ptr += align128((size_t)Vd * 4); }
    }
    cpx<R> *sR = (cpx<R> *)ptr;   ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));   // even half-field
    cpx<R> *sT = (cpx<R> *)ptr;   ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));   // odd half-field
    cpx<R> *sRo = (cpx<R> *)ptr;  ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));   // rho_o after inflow
    R *sRed = (R *)ptr;           ptr += align128((size_t)sap_red_elems(Vh) * sizeof(R));
    uint64_t *bar = (uint64_t *)ptr;  // [0]: links and clover staged, [1]: face slots staged
    // the face slots are staged over the odd half-fields sT and sRo (free at
    // the start of a visit) when they fit there; in FP32 only (FP64 would hold
    // the odd residual in registers meanwhile, and spill)
    cpx<R> *sF = sT;
    const uint32_t fbytes = (uint32_t)(6 * g.nf * sizeof(cpx<R>));
    const bool stage_faces = sizeof(R) == 4 && fbytes <= 2 * align128((size_t)12 * Vh * sizeof(cpx<R>));

    if (i == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
        // into L2 ahead of use (none of it is written by the previous half-sweep):
        // the clover blocks when they are read from global memory, and this
        // domain's residual and accumulated output
        if (!STC) {
            prefetch_l2(a.C.p + (int64_t)d * 36 * Vd, (uint32_t)(36 * Vd * sizeof(typename SC::T2)));
            if (SC::kScaled) prefetch_l2(a.C.scale + (int64_t)d * Vd, (uint32_t)(Vd * 4));
        }
        prefetch_l2(a.rho.p + (int64_t)d * 12 * Vd, (uint32_t)(12 * Vd * sizeof(typename SS::T2)));
        if (!a.first_psi) prefetch_l2(a.psi.p + (int64_t)d * 12 * Vd, (uint32_t)(12 * Vd * sizeof(typename SP::T2)));
    }
    __syncthreads();

    // stage the domain's links and clover blocks
    if (STL || STC) {
        if (i == 0) {
            uint32_t lb = STL ? (uint32_t)(36 * Vd * sizeof(typename SL::T2)) : 0;
            uint32_t cb = STC ? (uint32_t)(36 * Vd * sizeof(typename SC::T2)) : 0;
            uint32_t sb = (STC && SC::kScaled) ? (uint32_t)(Vd * 4) : 0;
            mbar_arrive_expect_tx(bar, lb + cb + sb);
            if (STL) bulk_g2s_chunked(sL, a.U.p + (int64_t)d * 36 * Vd, lb, bar);
            if (STC) bulk_g2s_chunked(sC, a.C.p + (int64_t)d * 36 * Vd, cb, bar);
            if (STC && SC::kScaled) bulk_g2s_chunked(sCs, a.C.scale + (int64_t)d * Vd, sb, bar);
        }
    }

    // neighbour slots and face indices of this thread's two sites, kept in
    // registers; the domain's neighbouring domains in shared memory
    uint16_t nbe[8], nbo[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        nbe[k] = __ldg(g.nbl + se * 8 + k);
        nbo[k] = __ldg(g.nbl + so * 8 + k);
    }
    const uint32_t fce = __ldg(g.fcoord + se), fco = __ldg(g.fcoord + so);
    __shared__ int sNbd[8];
    if (i < 8) sNbd[i] = __ldg(g.nbd + d * 8 + i);

    SapBlock<R, SL, SC, SS, SP, STL, STC> B{a, g, d, Vd, Vh, sL, sC, sCs};
    const R kappa = a.kappa;
    const int nwarps = (Vh + 31) / 32;
    const bool full_warps = (Vh % 32) == 0;
    const int nphase = 3 + 2 * a.nmr;

    // This domain's residual and output were last written by this colour's
    // previous half-sweep, two launches back.  Every half-sweep lets its
    // dependent start only after its own wait below, so that launch has
    // finished by now and the residual of the first right-hand side can be
    // read before the wait.  The face slots come from the previous launch.
    // (In FP32: holding it across the wait in FP64 would spill.)
    constexpr bool kEarly = sizeof(R) == 4;
    cpx<R> v[12], vo[12];
    if (kEarly) {
        load_sp<R, SS>(a.rho, 0, 0, d, se, Vd, v);
        load_sp<R, SS>(a.rho, 0, 0, d, so, Vd, vo);
    }
    pdl_wait();  // the previous half-sweep (other colour) has finished: its face slots are visible
    pdl_launch_dependents();
    for (int rr = 0; rr < a.nrhs; rr++) {
        const int64_t rb = rr * a.rstride, sb = rr * a.sstride;

        if ((STL || STC) && rr == 0) {
            bool ok = mbar_wait_bounded(bar, 0, QDD_FIRST_WAIT_SPINS);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                // give the copies in flight a last bounded chance to land, then leave
                mbar_wait_bounded(bar, 0, 1u << 20);
                return;
            }
        }

        // residual of this domain plus the inflow of the other colour's last
        // corrections across the faces: rho += kappa * (hops that enter)
        const int64_t fr = rr * a.fstride;
        const cpx<R> *fd = a.face + fr + (int64_t)d * 6 * g.nf;
        if (a.gather && stage_faces) {
            // one bulk copy of this domain's face slots (written by the previous
            // half-sweep) instead of a dependent load per crossing hop
            if (i == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar + 1, fbytes);
                bulk_g2s_chunked(sF, fd, fbytes, bar + 1);
            }
            bool ok = mbar_wait_bounded(bar + 1, rr & 1, 1u << 22);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                mbar_wait_bounded(bar + 1, rr & 1, 1u << 20);
                return;
            }
            fd = sF;
        }
        // rho_e parks in sR until the setup phase, rho_o in sRo (once every
        // thread has read the staged face slots that overlap it)
        // (the two sites run through one copy of the face code: a loop with
        // element-wise selects, which keeps the kernel in the instruction cache)
        cpx<R> acc[12];
        if (rr > 0 || !kEarly) load_sp<R, SS>(a.rho, rb, sb, d, se, Vd, v);
        if (rr > 0 && kEarly) load_sp<R, SS>(a.rho, rb, sb, d, so, Vd, vo);
        const bool hold = a.gather && stage_faces;
        // FP64 unrolls both loops (its register arrays are twice as wide, and
        // the selects of the rolled form spill there)
        constexpr int kSiteUnroll = sizeof(R) == 8 ? 2 : 1;
#pragma unroll kSiteUnroll
        for (int par = 0; par < 2; par++) {
            const int s = par ? so : se;
            cpx<R> t[12];
            if (kEarly) {
#pragma unroll
                for (int k = 0; k < 12; k++) t[k] = par ? vo[k] : v[k];
            } else if (par) {
                load_sp<R, SS>(a.rho, rb, sb, d, so, Vd, t);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) t[k] = v[k];
            }
            if (a.gather) {
                uint16_t nb[8];
#pragma unroll
                for (int k = 0; k < 8; k++) nb[k] = par ? nbo[k] : nbe[k];
                auto lnk = [&](int mu, cpx<R> *u) { B.link(d, s, mu, u); };
                face_in(g, nb, par ? fco : fce, fd, lnk, acc);
#pragma unroll
                for (int k = 0; k < 12; k++) t[k] = t[k] + kappa * acc[k];
            }
            if (par == 0) {
#pragma unroll
                for (int k = 0; k < 12; k++) sR[k * Vh + i] = t[k];
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) vo[k] = t[k];
            }
        }
        if (hold) __syncthreads();
#pragma unroll
        for (int k = 0; k < 12; k++) sRo[k * Vh + i] = vo[k];

        // MR solution x_e in registers; the MR residual r lives in sR between
        // phases (read back where it is needed, which keeps it out of the
        // registers during the hop sums)
        cpx<R> x[12];
#pragma unroll
        for (int k = 0; k < 12; k++) x[k] = mk<R>(0, 0);

        for (int ph = 0; ph < nphase; ph++) {
            const int type = ph == 0 ? PH_SETUP_ODD
                             : ph == 1 ? PH_SETUP_EVEN
                             : ph == nphase - 1 ? PH_RECON_ODD
                             : ((ph & 1) ? PH_MR_EVEN : PH_MR_ODD);
            const int par = (type == PH_SETUP_EVEN || type == PH_MR_EVEN) ? 0 : 1;
            const int s = par ? so : se;

            // hop sum from the other parity's half-field (Dirichlet boundary)
            if (type != PH_SETUP_ODD) {
                uint16_t nb[8];
#pragma unroll
                for (int k = 0; k < 8; k++) nb[k] = par ? nbo[k] : nbe[k];
                B.inner_hops(s, nb, par ? sR : sT, par ? 0 : Vh, acc);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
            }

            // own operand and clover input
            //   setup-odd: A^-1 rho_o     mr-odd: A^-1 (-k acc)
            //   mr-even:   A r            recon:  A^-1 (rho_o + k acc)
            if (type == PH_SETUP_EVEN) {
                // r = rho_e + kappa acc; with nmr = 0 the reconstruction reads x = 0
                // and r is the final residual
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    v[k] = sR[k * Vh + i] + kappa * acc[k];
                    sR[k * Vh + i] = a.nmr > 0 ? v[k] : x[k];
                }
                if (a.nmr == 0) store_sp<R, SS>(a.rho, rb, sb, d, se, Vd, v);
                __syncthreads();
                continue;
            }
            cpx<R> r[12];  // MR residual (mr-even)
            if (type == PH_MR_EVEN) {
#pragma unroll
                for (int k = 0; k < 12; k++) r[k] = sR[k * Vh + i];
            }
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cpx<R> own = type == PH_MR_EVEN ? r[k] : (type == PH_MR_ODD ? mk<R>(0, 0) : sRo[k * Vh + i]);
                R ka = type == PH_MR_EVEN || type == PH_SETUP_ODD ? (R)0 : (type == PH_MR_ODD ? -kappa : kappa);
                v[k] = own + ka * acc[k];
            }
            cpx<R> c[12];
            B.clover(s, v, c);

            if (type == PH_MR_EVEN) {
                // p = A r + kappa acc ; alpha = <p,r>/<p,p> ; x += alpha r ; r -= alpha p
                R pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    c[k] = c[k] + kappa * acc[k];
                    pr_re = fma(c[k].re, r[k].re, pr_re);
                    pr_re = fma(c[k].im, r[k].im, pr_re);
                    pr_im = fma(c[k].re, r[k].im, pr_im);
                    pr_im = fma(-c[k].im, r[k].re, pr_im);
                    pp = fma(c[k].re, c[k].re, pp);
                    pp = fma(c[k].im, c[k].im, pp);
                }
                if (full_warps) {
                    pr_re = warp_sum(pr_re);
                    pr_im = warp_sum(pr_im);
                    pp = warp_sum(pp);
                    if ((i & 31) == 0 && QDD_IN_RANGE((i >> 5) * 4 + 2, 0, sap_red_elems(Vh))) {
                        sRed[(i >> 5) * 4 + 0] = pr_re;
                        sRed[(i >> 5) * 4 + 1] = pr_im;
                        sRed[(i >> 5) * 4 + 2] = pp;
                    }
                } else {
                    // partial warp: per-thread partials, summed in order below
                    if (QDD_IN_RANGE(i * 3 + 2, 0, sap_red_elems(Vh))) {
                        sRed[i * 3 + 0] = pr_re;
                        sRed[i * 3 + 1] = pr_im;
                        sRed[i * 3 + 2] = pp;
                    }
                }
                __syncthreads();
                R tr = 0, ti_ = 0, tp = 0;
                if (full_warps) {
                    for (int w = 0; w < nwarps; w++) {
                        tr += sRed[w * 4 + 0];
                        ti_ += sRed[w * 4 + 1];
                        tp += sRed[w * 4 + 2];
                    }
                } else {
                    for (int w = 0; w < Vh; w++) {
                        tr += sRed[w * 3 + 0];
                        ti_ += sRed[w * 3 + 1];
                        tp += sRed[w * 3 + 2];
                    }
                }
                cpx<R> alpha = tp > (R)0 ? mk<R>(tr / tp, ti_ / tp) : mk<R>(0, 0);
                const bool last = ph == nphase - 2;
                // sR was last read before this phase's hop sum completed on
                // every thread (barrier above); sRed is rewritten only after
                // the next phase's barrier
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    cfma(x[k], alpha, r[k]);
                    r[k] = r[k] - alpha * c[k];
                    sR[k * Vh + i] = last ? x[k] : r[k];
                }
                if (last) store_sp<R, SS>(a.rho, rb, sb, d, se, Vd, r);  // final residual, even site
            } else {
                // setup-odd / mr-odd: t_o -> sT; reconstruction: x_o -> sT
#pragma unroll
                for (int k = 0; k < 12; k++) sT[k * Vh + i] = c[k];
            }
            __syncthreads();
        }

        // Outputs of the visit, after the phase loop (kept out of its body so
        // that the loop stays in the instruction cache): the correction
        // delta = (x_e in sR, x_o in sT) pushed across the faces, psi += delta,
        // and the odd residual, now zero.  The even residual was stored by the
        // last MR step.
#pragma unroll kSiteUnroll
        for (int par = 0; par < 2; par++) {
            const int s = par ? so : se;
            const cpx<R> *src = par ? sT : sR;
            cpx<R> dl[12];
#pragma unroll
            for (int k = 0; k < 12; k++) dl[k] = src[k * Vh + i];
            uint16_t nb[8];
#pragma unroll
            for (int k = 0; k < 8; k++) nb[k] = par ? nbo[k] : nbe[k];
            B.face_out(s, nb, par ? fco : fce, sNbd, dl, a.face + fr);
            if (a.first_psi) {
                store_sp<R, SP>(a.psi, rb, sb, d, s, Vd, dl);
            } else {
                cpx<R> q[12];
                load_sp<R, SP>(a.psi, rb, sb, d, s, Vd, q);
#pragma unroll
                for (int k = 0; k < 12; k++) q[k] = q[k] + dl[k];
                store_sp<R, SP>(a.psi, rb, sb, d, s, Vd, q);
            }
            if (par) {
#pragma unroll
                for (int k = 0; k < 12; k++) dl[k] = mk<R>(0, 0);
                store_sp<R, SS>(a.rho, rb, sb, d, s, Vd, dl);
            }
        }
        if (rr + 1 < a.nrhs) __syncthreads();  // sT and sRo are restaged for the next source
    }
}

// ------------------------------------------------- paired-thread form
//
// The same domain visit with two threads per even/odd site pair (FP32
// arithmetic, links and clover staged, half-fields of whole warps).  The
// first Vh threads form half 0, the others half 1 (whole warps, so every
// branch on the half is uniform in a warp).  Half hb owns clover block hb,
// i.e. the six components of spins (2hb, 2hb+1) of every vector of the MR
// iteration, and runs the hops of directions 2hb and 2hb+1.  Its partial
// hop sum holds all twelve components, its own six first; the other six go
// to the partner thread through shared memory: in the even phases through
// the buffer that held the inflowing odd residual (which stays in registers
// for the visit), in the odd phases through the odd half-field, whose
// content the previous even phase has consumed.  Face inflow and outflow and
// the global loads and stores run one site per thread: half 0 the even site,
// half 1 the odd site.  The kernel runs twice the warps of the one-thread
// form in the same shared memory, at 128 registers per thread, so more
// warps cover each other's shared-memory and arithmetic latencies; it also
// executes more instructions per site (each thread's clover block in scalar
// FMAs, the exchange).  With FP32 links, where the one-thread form holds a
// single 4-warp CTA per SM, that pays (32^3x64: 0.647 against 0.927 ms per
// half-sweep); with 16-bit links, two one-thread CTAs share an SM and the
// paired form is not faster (48^3x96 BF16: 2.40 against 2.29 ms).  The two
// partial sums are added last, and the MR dot products run over six
// components per thread, so results agree with the one-thread form to
// rounding, not bit for bit.
template <typename SL, typename SC, typename SS, typename SP, int MAXT, int MINB, int SHAPE>
__global__ void __launch_bounds__(MAXT, MINB) k_sap_pair(const SapArgs<float, SL, SC, SS, SP> a)
{
    using R = float;
    extern __shared__ __align__(128) unsigned char smem[];
    const Geom g = sap_geom<SHAPE>(a.g);
    const int Vd = g.Vd, Vh = g.Vh;
    const int i = threadIdx.x;
    const int hb = i >= Vh ? 1 : 0;      // the half (uniform in a warp)
    const int p = i - hb * Vh;           // the site pair
    const int mb = 6 * hb, ob = 6 - mb;  // first of the own / the partner's six components
    const int bx = blockIdx.x;
    const int d = sap_domain(a, g.Nd2, bx);
    const int se = p, so = Vh + p, sown = hb ? so : se;

    unsigned char *ptr = smem;
    typename SL::T2 *sL = (typename SL::T2 *)ptr;
    ptr += align128((size_t)36 * Vd * sizeof(typename SL::T2));
    typename SC::T2 *sC = (typename SC::T2 *)ptr;
    ptr += align128((size_t)36 * Vd * sizeof(typename SC::T2));
    float *sCs = nullptr;
    if (SC::kScaled) { sCs = (float *)ptr; ptr += align128((size_t)Vd * 4); }
    cpx<R> *sR = (cpx<R> *)ptr;  ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));  // even half-field
    cpx<R> *sT = (cpx<R> *)ptr;  ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));  // odd half-field
    cpx<R> *sX = (cpx<R> *)ptr;  ptr += align128((size_t)12 * Vh * sizeof(cpx<R>));  // rho_o, then exchange
    R *sRed = (R *)ptr;          ptr += align128((size_t)sap_red_elems(Vh) * sizeof(R));
    uint64_t *bar = (uint64_t *)ptr;
    cpx<R> *sF = sT;  // staged face slots, over sT and sX
    const uint32_t fbytes = (uint32_t)(6 * g.nf * sizeof(cpx<R>));
    const bool stage_faces = fbytes <= 2 * align128((size_t)12 * Vh * sizeof(cpx<R>));

    if (i == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
        prefetch_l2(a.rho.p + (int64_t)d * 12 * Vd, (uint32_t)(12 * Vd * sizeof(typename SS::T2)));
        if (!a.first_psi) prefetch_l2(a.psi.p + (int64_t)d * 12 * Vd, (uint32_t)(12 * Vd * sizeof(typename SP::T2)));
    }
    __syncthreads();
    if (i == 0) {
        const uint32_t lb = (uint32_t)(36 * Vd * sizeof(typename SL::T2));
        const uint32_t cb = (uint32_t)(36 * Vd * sizeof(typename SC::T2));
        const uint32_t sb = SC::kScaled ? (uint32_t)(Vd * 4) : 0;
        mbar_arrive_expect_tx(bar, lb + cb + sb);
        bulk_g2s_chunked(sL, a.U.p + (int64_t)d * 36 * Vd, lb, bar);
        bulk_g2s_chunked(sC, a.C.p + (int64_t)d * 36 * Vd, cb, bar);
        if (SC::kScaled) bulk_g2s_chunked(sCs, a.C.scale + (int64_t)d * Vd, sb, bar);
    }

    // the neighbour entries of the two directions of this half, for the
    // even and the odd site of the pair
    uint16_t nbe[4], nbo[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        nbe[k] = __ldg(g.nbl + se * 8 + 4 * hb + k);
        nbo[k] = __ldg(g.nbl + so * 8 + 4 * hb + k);
    }
    __shared__ int sNbd[8];
    if (i < 8) sNbd[i] = __ldg(g.nbd + d * 8 + i);

    SapBlock<R, SL, SC, SS, SP, true, true, true> B{a, g, d, Vd, Vh, sL, sC, sCs};
    const R kappa = a.kappa;
    const int nwarps = 2 * Vh / 32;
    const int nphase = 3 + 2 * a.nmr;

    // the residual of this thread's site: read before the wait, as in the
    // one-thread form (written two launches back)
    cpx<R> v[12];
    load_sp<R, SS>(a.rho, 0, 0, d, sown, Vd, v);
    pdl_wait();
    pdl_launch_dependents();
    for (int rr = 0; rr < a.nrhs; rr++) {
        const int64_t rb = rr * a.rstride, sb = rr * a.sstride;
        if (rr == 0) {
            bool ok = mbar_wait_bounded(bar, 0, QDD_FIRST_WAIT_SPINS);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                mbar_wait_bounded(bar, 0, 1u << 20);
                return;
            }
        }
        const int64_t fr = rr * a.fstride;
        const cpx<R> *fd = a.face + fr + (int64_t)d * 6 * g.nf;
        const bool hold = a.gather && stage_faces;
        if (hold) {
            if (i == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar + 1, fbytes);
                bulk_g2s_chunked(sF, fd, fbytes, bar + 1);
            }
            bool ok = mbar_wait_bounded(bar + 1, rr & 1, 1u << 22);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                mbar_wait_bounded(bar + 1, rr & 1, 1u << 20);
                return;
            }
            fd = sF;
        }
        if (rr > 0) load_sp<R, SS>(a.rho, rb, sb, d, sown, Vd, v);
        // residual plus the inflow across the faces, one site per thread
        if (a.gather) {
            uint16_t nb[8];
#pragma unroll
            for (int k = 0; k < 8; k++) nb[k] = __ldg(g.nbl + sown * 8 + k);
            cpx<R> acc[12];
            auto lnk = [&](int mu, cpx<R> *u) { B.link(d, sown, mu, u); };
            face_in(g, nb, __ldg(g.fcoord + sown), fd, lnk, acc);
#pragma unroll
            for (int k = 0; k < 12; k++) v[k] = v[k] + kappa * acc[k];
        }
        if (hold) __syncthreads();  // every thread has read the staged slots
        {
            hf_store<12, true>(hb ? sX : sR, 0, p, Vh, v);
        }
        __syncthreads();

        // own components of rho_o (for the whole visit) and of x_e
        cpx<R> ro[6], x[6];
#pragma unroll
        for (int j = 0; j < 6; j++) x[j] = mk<R>(0, 0);
        hf_load<6, true>(sX, mb, p, Vh, ro);

        for (int ph = 0; ph < nphase; ph++) {
            const int type = ph == 0 ? PH_SETUP_ODD
                             : ph == 1 ? PH_SETUP_EVEN
                             : ph == nphase - 1 ? PH_RECON_ODD
                             : ((ph & 1) ? PH_MR_EVEN : PH_MR_ODD);
            const int par = (type == PH_SETUP_EVEN || type == PH_MR_EVEN) ? 0 : 1;
            const int s = par ? so : se;

            // own components of the hop sum from the other parity's half-field
            cpx<R> hs[6];
            if (type != PH_SETUP_ODD) {
                cpx<R> acc[12];  // own six components first
#pragma unroll
                for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
                const cpx<R> *src = par ? sR : sT;
                const int off = par ? 0 : Vh;
                uint16_t e[4];
#pragma unroll
                for (int k = 0; k < 4; k++) e[k] = par ? nbo[k] : nbe[k];
                if (hb == 0) {
                    B.template inner_dir_e<0>(s, e[0], e[1], src, off, acc);
                    B.template inner_dir_e<1>(s, e[2], e[3], src, off, acc);
                } else {
                    B.template inner_dir_e<2, true>(s, e[0], e[1], src, off, acc);
                    B.template inner_dir_e<3, true>(s, e[2], e[3], src, off, acc);
                }
                cpx<R> *xb = par ? sT : sX;
                hf_store<6, true>(xb, ob, p, Vh, acc + 6);
                __syncthreads();
                hf_load<6, true>(xb, mb, p, Vh, hs);
#pragma unroll
                for (int j = 0; j < 6; j++) hs[j] = acc[j] + hs[j];
            } else {
#pragma unroll
                for (int j = 0; j < 6; j++) hs[j] = mk<R>(0, 0);
            }

            if (type == PH_SETUP_EVEN) {
                // r = rho_e + kappa acc (with nmr = 0 also the final residual, kept in sX)
                cpx<R> rj[6];
                hf_load<6, true>(sR, mb, p, Vh, rj);
#pragma unroll
                for (int j = 0; j < 6; j++) rj[j] = rj[j] + kappa * hs[j];
                if (a.nmr > 0) {
                    hf_store<6, true>(sR, mb, p, Vh, rj);
                } else {
                    hf_store<6, true>(sR, mb, p, Vh, x);
                    hf_store<6, true>(sX, mb, p, Vh, rj);
                }
                __syncthreads();
                continue;
            }
            cpx<R> r[6];
            if (type == PH_MR_EVEN) hf_load<6, true>(sR, mb, p, Vh, r);
            cpx<R> w[6];
#pragma unroll
            for (int j = 0; j < 6; j++) {
                cpx<R> own = type == PH_MR_EVEN ? r[j] : (type == PH_MR_ODD ? mk<R>(0, 0) : ro[j]);
                R ka = type == PH_MR_EVEN || type == PH_SETUP_ODD ? (R)0 : (type == PH_MR_ODD ? -kappa : kappa);
                w[j] = own + ka * hs[j];
            }
            cpx<R> c[6];
            B.clover_blk(s, hb, w, c);

            if (type == PH_MR_EVEN) {
                R pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    c[j] = c[j] + kappa * hs[j];
                    pr_re = fma(c[j].re, r[j].re, pr_re);
                    pr_re = fma(c[j].im, r[j].im, pr_re);
                    pr_im = fma(c[j].re, r[j].im, pr_im);
                    pr_im = fma(-c[j].im, r[j].re, pr_im);
                    pp = fma(c[j].re, c[j].re, pp);
                    pp = fma(c[j].im, c[j].im, pp);
                }
                pr_re = warp_sum(pr_re);
                pr_im = warp_sum(pr_im);
                pp = warp_sum(pp);
                if ((i & 31) == 0 && QDD_IN_RANGE((i >> 5) * 4 + 2, 0, sap_red_elems(Vh))) {
                    sRed[(i >> 5) * 4 + 0] = pr_re;
                    sRed[(i >> 5) * 4 + 1] = pr_im;
                    sRed[(i >> 5) * 4 + 2] = pp;
                }
                __syncthreads();
                R tr = 0, ti_ = 0, tp = 0;
                for (int wv = 0; wv < nwarps; wv++) {
                    tr += sRed[wv * 4 + 0];
                    ti_ += sRed[wv * 4 + 1];
                    tp += sRed[wv * 4 + 2];
                }
                const cpx<R> alpha = tp > (R)0 ? mk<R>(tr / tp, ti_ / tp) : mk<R>(0, 0);
                const bool last = ph == nphase - 2;
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    cfma(x[j], alpha, r[j]);
                    r[j] = r[j] - alpha * c[j];
                }
                if (last) {
                    hf_store<6, true>(sR, mb, p, Vh, x);
                    hf_store<6, true>(sX, mb, p, Vh, r);  // the final residual
                } else {
                    hf_store<6, true>(sR, mb, p, Vh, r);
                }
            } else {
                // setup-odd / mr-odd: t_o; reconstruction: x_o (own components)
                hf_store<6, true>(sT, mb, p, Vh, c);
            }
            __syncthreads();
        }

        // outputs of the visit, one site per thread: the correction delta
        // (x_e in sR, x_o in sT) pushed across the faces, psi += delta; the
        // residual: the final MR residual (in sX) on the even site, zero on
        // the odd site
        {
            const cpx<R> *src = hb ? sT : sR;
            cpx<R> dl[12];
            hf_load<12, true>(src, 0, p, Vh, dl);
            uint16_t nb[8];
#pragma unroll
            for (int k = 0; k < 8; k++) nb[k] = __ldg(g.nbl + sown * 8 + k);
            B.face_out(sown, nb, __ldg(g.fcoord + sown), sNbd, dl, a.face + fr);
            if (a.first_psi) {
                store_sp<R, SP>(a.psi, rb, sb, d, sown, Vd, dl);
            } else {
                cpx<R> q[12];
                load_sp<R, SP>(a.psi, rb, sb, d, sown, Vd, q);
#pragma unroll
                for (int k = 0; k < 12; k++) q[k] = q[k] + dl[k];
                store_sp<R, SP>(a.psi, rb, sb, d, sown, Vd, q);
            }
            if (hb) {
#pragma unroll
                for (int k = 0; k < 12; k++) dl[k] = mk<R>(0, 0);
            } else {
                hf_load<12, true>(sX, 0, p, Vh, dl);
            }
            store_sp<R, SS>(a.rho, rb, sb, d, sown, Vd, dl);
        }
        if (rr + 1 < a.nrhs) __syncthreads();  // sR, sT and sX are restaged for the next source
    }
}

// ------------------------------------------------------------ face inflow
//
// Applies the pending face slots of the domains of one colour to their
// residual, without a block solve (brings the residual of the next colour up
// to date after the last half-sweep).  One thread per site.

template <typename R, typename SL, typename SS>
__global__ void __launch_bounds__(128) k_sap_face_apply(const Geom g, const Field<SL> U, Field<SS> rho,
                                                        const cpx<R> *face, int64_t rstride, int64_t sstride,
                                                        int64_t fstride, R kappa, int colour, int nrhs)
{
    const int Vd = g.Vd;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.Nd2 * Vd) return;
    const int d = colour * g.Nd2 + gi / Vd, s = gi % Vd;
    uint16_t nb[8];
    bool any = false;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        nb[k] = __ldg(g.nbl + s * 8 + k);
        any |= (nb[k] & kCross) != 0;
    }
    if (!any) return;  // interior site: no hop enters from another domain
    auto lnk = [&](int mu, cpx<R> *u) {
        const typename SL::T2 *p = U.p + ((int64_t)d * 36 + mu * 9) * Vd + s;
#pragma unroll
        for (int k = 0; k < 9; k++) u[k] = ld_c<R>(p + (int64_t)k * Vd);
    };
    for (int rr = 0; rr < nrhs; rr++) {
        cpx<R> acc[12], v[12];
        face_in(g, nb, __ldg(g.fcoord + s), face + rr * fstride + (int64_t)d * 6 * g.nf, lnk, acc);
        load_sp<R, SS>(rho, rr * rstride, rr * sstride, d, s, Vd, v);
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = v[k] + kappa * acc[k];
        store_sp<R, SS>(rho, rr * rstride, rr * sstride, d, s, Vd, v);
    }
}

// ---------------------------------------------------------------- launch

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC, int MAXT = 256,
          int MINB = 1, int SHAPE = 0>
static qdd_status run_sap(Gauge *g, const SapArgs<R, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl, bool timed)
{
    const HostGeom &hg = g->hg;
    size_t smem = sap_smem_layout<R, SL, SC>(hg.Vd, STL, STC);
    auto kern = k_sap<R, SL, SC, SS, SP, STL, STC, MAXT, MINB, SHAPE>;
    static thread_local size_t configured = 0;
    if (configured < smem) {
        QDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (MINB > 1)  // room for MINB CTAs' shared memory on an SM
            QDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        configured = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblocks);
    cfg.blockDim = dim3(hg.Vh);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    LaunchScope ls(g->ctx->timer, K_SAP, s, timed);
    QDD_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return QDD_OK;
}

template <typename SL, typename SC, typename SS, typename SP, int MAXT, int MINB, int SHAPE>
static qdd_status run_sap_pair(Gauge *g, const SapArgs<float, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl,
                               bool timed)
{
    const HostGeom &hg = g->hg;
    size_t smem = sap_smem_layout<float, SL, SC>(hg.Vd, true, true);
    auto kern = k_sap_pair<SL, SC, SS, SP, MAXT, MINB, SHAPE>;
    static thread_local size_t configured = 0;
    if (configured < smem) {
        QDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        QDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        configured = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblocks);
    cfg.blockDim = dim3(2 * hg.Vh);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    LaunchScope ls(g->ctx->timer, K_SAP, s, timed);
    QDD_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return QDD_OK;
}

static size_t smem_limit()
{
    static size_t lim = 0;
    if (!lim) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        lim = (size_t)v;
    }
    return lim;
}

static size_t smem_per_sm()
{
    static size_t lim = 0;
    if (!lim) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        lim = (size_t)v;
    }
    return lim;
}

// Links are staged in shared memory, then the Schwarz clover when it fits too.
template <typename R, typename SL, typename SC, typename SS, typename SP>
static qdd_status dispatch_staging(Gauge *g, const SapArgs<R, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl,
                                   bool timed, int gather_only)
{
    const HostGeom &hg = g->hg;
    if (gather_only) {
        const int n = hg.Nd2 * hg.Vd;
        g->ctx->timer.count(K_OTHER);
        k_sap_face_apply<R, SL, SS><<<(n + 127) / 128, 128, 0, s>>>(a.g, a.U, a.rho, a.face, a.rstride, a.sstride,
                                                                     a.fstride, a.kappa, a.colour, a.nrhs);
        QDD_CUDA(cudaGetLastError());
        return QDD_OK;
    }
    const int Vd = hg.Vd;
    const size_t lim = smem_limit() - 128;  // the kernel's static shared memory
    int shape = (hg.dom[1] == 4 && hg.dom[2] == 4 && hg.dom[3] == 4) ? (hg.dom[0] == 4 ? 1 : (hg.dom[0] == 8 ? 2 : 0)) : 0;
    if (shape) {  // the fixed form's constants (sap_geom) must be the geometry's
        const int fx = Vd / hg.dom[0], fo = Vd / 4;
        const int foff[8] = {0, fx, 2 * fx, 2 * fx + fo, 2 * fx + 2 * fo, 2 * fx + 3 * fo, 2 * fx + 4 * fo,
                             2 * fx + 5 * fo};
        bool same = hg.nf == 2 * (fx + 3 * fo) && hg.Vd == (shape == 1 ? 256 : 512);
        for (int k = 0; k < 8; k++) same = same && hg.foff[k] == foff[k];
        if (!same) shape = 0;
    }
    // the occupancy form: links staged, clover read through the cache, three
    // CTAs per SM (FP32 arithmetic, domains of at most 256 sites)
    if constexpr (sizeof(R) == 4) {
        if (g->sap_variant == 1 && hg.Vh <= 128 && 3 * (sap_smem_layout<R, SL, SC>(Vd, true, false) + 128) <= 3 * lim &&
            3 * (sap_smem_layout<R, SL, SC>(Vd, true, false) + 1024) <= smem_per_sm())
            return run_sap<R, SL, SC, SS, SP, true, false, 128, 3>(g, a, s, pdl, timed);
    }
    // the paired-thread form: FP32 arithmetic, links and clover staged,
    // half-fields of whole warps, at most 512 threads.  The default with FP32
    // links, where the one-thread form runs one CTA of Vh threads per SM (4^4
    // domains, 32^3x64: 0.647 against 0.927 ms per half-sweep); with 16-bit
    // links two one-thread CTAs share an SM and the paired form, with more
    // instructions per site, is no faster (48^3x96 BF16: 2.40 against 2.29 ms).
    if constexpr (sizeof(R) == 4) {
        const bool pair = g->sap_variant == 3 || (g->sap_variant == 0 && std::is_same<SL, StF32>::value);
        if (pair && hg.Vh % 32 == 0 && 2 * hg.Vh <= 512 && sap_smem_layout<R, SL, SC>(Vd, true, true) <= lim) {
            constexpr int kMinb = sizeof(typename SL::T2) == 4 ? 2 : 1;  // 16-bit: two 4^4 domains per SM
            if (shape == 1) return run_sap_pair<SL, SC, SS, SP, 256, kMinb, 1>(g, a, s, pdl, timed);
            if (shape == 2) return run_sap_pair<SL, SC, SS, SP, 512, 1, 2>(g, a, s, pdl, timed);
            return run_sap_pair<SL, SC, SS, SP, 512, 1, 0>(g, a, s, pdl, timed);
        }
    }
    if (sap_smem_layout<R, SL, SC>(Vd, true, true) <= lim) {
        // 4^4 domains (the 16-bit workloads' shape): the shape fixed at compile time
        if constexpr (sizeof(R) == 4 && !std::is_same<SL, StF32>::value)
            if (shape == 1 && g->sap_variant == 0)
                return run_sap<R, SL, SC, SS, SP, true, true, 128, 2, 1>(g, a, s, pdl, timed);
        return run_sap<R, SL, SC, SS, SP, true, true>(g, a, s, pdl, timed);
    }
    if (sap_smem_layout<R, SL, SC>(Vd, true, false) <= lim) {
        // 8x4^3 domains with FP32 links (the clover does not fit): the shape fixed at compile time
        if constexpr (sizeof(R) == 4 && std::is_same<SL, StF32>::value)
            if (shape == 2 && g->sap_variant == 0)
                return run_sap<R, SL, SC, SS, SP, true, false, 256, 1, 2>(g, a, s, pdl, timed);
        return run_sap<R, SL, SC, SS, SP, true, false>(g, a, s, pdl, timed);
    }
    if (sap_smem_layout<R, SL, SC>(Vd, false, false) <= lim)
        return run_sap<R, SL, SC, SS, SP, false, false>(g, a, s, pdl, timed);
    set_error("domain of %d sites does not fit in shared memory", Vd);
    return QDD_EINVAL;
}

// the first wait's poll limit on the current device (QDD_CHECK builds)
qdd_status set_first_wait_spins_sap(unsigned spins)
{
#ifdef QDD_CHECK
    QDD_CUDA(cudaMemcpyToSymbol(g_first_wait_spins, &spins, sizeof(spins)));
    QDD_CUDA(cudaDeviceSynchronize());
    return QDD_OK;
#else
    (void)spins;
    set_error("this library was built without range checks (QDD_CHECK)");
    return QDD_EINVAL;
#endif
}

// out-of-range indices the kernels of this file have skipped (QDD_CHECK builds)
unsigned long long check_hits_sap()
{
#ifdef QDD_CHECK
    unsigned long long h = 0;
    if (cudaMemcpyFromSymbol(&h, g_check_hits, sizeof(h)) != cudaSuccess) return ~0ull;
    return h;
#else
    return 0;
#endif
}

size_t sap_face_bytes(const HostGeom &hg, qdd_prec prec, int nrhs)
{
    const size_t e = prec == QDD_PREC_F64 ? sizeof(double2) : sizeof(float2);
    return (size_t)hg.Nd * 6 * hg.nf * e * (size_t)nrhs;
}

size_t sap_smem_bytes(const HostGeom &hg, qdd_prec prec, bool stl, bool stc)
{
    switch (prec) {
    case QDD_PREC_F64: return sap_smem_layout<double, StF64, StF64>(hg.Vd, stl, stc);
    case QDD_PREC_F32: return sap_smem_layout<float, StF32, StF32>(hg.Vd, stl, stc);
    case QDD_PREC_F16S: return sap_smem_layout<float, StF16, StF16>(hg.Vd, stl, stc);
    case QDD_PREC_H16: return sap_smem_layout<float, StF16, StF16>(hg.Vd, stl, stc);
    default: return sap_smem_layout<float, StBF16, StBF16>(hg.Vd, stl, stc);
    }
}

qdd_status launch_sap_halfsweep(Gauge *g, qdd_prec prec, const SapBuffers &b, int colour, int nmr, int nrhs,
                                int first_psi, int gather, int gather_only, int *d_err, cudaStream_t s, bool pdl,
                                bool timed, int part)
{
    QDD_TRY(ensure_copy(g, prec, s));
    const int64_t rs = (int64_t)g->hg.V * 12, ss = g->hg.V, fs = (int64_t)g->hg.Nd * 6 * g->hg.nf;
    // part 1: the first and last t-block's domains of the colour; part 2: the others
    const int half = g->hg.nb[0] * g->hg.nb[1] * g->hg.nb[2] / 2, nd2 = g->hg.Nd2;
    const int dfirst = part == 2 ? half : 0;
    const int nsplit = part == 1 ? half : (part == 2 ? nd2 - 2 * half : nd2);
    const int dskip = part == 1 ? nd2 - 2 * half : 0;
    const int nblocks = part == 1 ? 2 * half : nsplit;
    if (nblocks == 0) return QDD_OK;  // a slab of two t-blocks has no interior
    PrecCopy &c = g->copies[prec];
    switch (prec) {
    case QDD_PREC_F64: {
        SapArgs<double, StF64, StF64, StF64, StF64> a{
            g->geom, {g->links64.as<double2>(), nullptr}, {g->sclov64.as<double2>(), nullptr},
            {(double2 *)b.rho, nullptr}, (cpx<double> *)b.face, {(double2 *)b.psi, nullptr},
            rs, ss, fs, g->kappa, colour, nmr, nrhs, first_psi, gather, d_err, dfirst, nsplit, dskip, nblocks};
        return dispatch_staging(g, a, s, pdl, timed, gather_only);
    }
    case QDD_PREC_F32: {
        SapArgs<float, StF32, StF32, StF32, StF32> a{
            g->geom, {c.links.as<float2>(), nullptr}, {c.sclov.as<float2>(), nullptr},
            {(float2 *)b.rho, nullptr}, (cpx<float> *)b.face, {(float2 *)b.psi, nullptr},
            rs, ss, fs, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, d_err, dfirst, nsplit, dskip, nblocks};
        return dispatch_staging(g, a, s, pdl, timed, gather_only);
    }
    case QDD_PREC_F16S: {
        SapArgs<float, StF16, StF16, StF16, StF32> a{
            g->geom, {c.links.as<__half2>(), nullptr}, {c.sclov.as<__half2>(), c.sclov_s.as<float>()},
            {(__half2 *)b.rho, b.rho_s}, (cpx<float> *)b.face, {(float2 *)b.psi, nullptr},
            rs, ss, fs, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, d_err, dfirst, nsplit, dskip, nblocks};
        return dispatch_staging(g, a, s, pdl, timed, gather_only);
    }
    case QDD_PREC_H16: {
        PrecCopy &h = g->copies[QDD_PREC_F16S];
        SapArgs<float, StF16, StF16, StF32, StF32> a{
            g->geom, {h.links.as<__half2>(), nullptr}, {h.sclov.as<__half2>(), h.sclov_s.as<float>()},
            {(float2 *)b.rho, nullptr}, (cpx<float> *)b.face, {(float2 *)b.psi, nullptr},
            rs, ss, fs, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, d_err, dfirst, nsplit, dskip, nblocks};
        return dispatch_staging(g, a, s, pdl, timed, gather_only);
    }
    case QDD_PREC_BF16S: {
        SapArgs<float, StBF16, StBF16, StBF16, StF32> a{
            g->geom, {c.links.as<__nv_bfloat162>(), nullptr}, {c.sclov.as<__nv_bfloat162>(), c.sclov_s.as<float>()},
            {(__nv_bfloat162 *)b.rho, b.rho_s}, (cpx<float> *)b.face, {(float2 *)b.psi, nullptr},
            rs, ss, fs, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, d_err, dfirst, nsplit, dskip, nblocks};
        return dispatch_staging(g, a, s, pdl, timed, gather_only);
    }
    default: break;
    }
    set_error("invalid preconditioner precision %d", (int)prec);
    return QDD_EINVAL;
}

}  // namespace qdd
