// Schwarz alternating procedure (multiplicative Schwarz), one colour half-sweep
// per launch (arXiv:1502.04025, Sec. 3.1; Sec. 3.5: cores synchronise only
// after an MR block solve, here the kernel boundary).
//
// One CTA per domain Lambda of the colour being swept, one thread per
// even/odd site pair.  The domain's links and Schwarz clover blocks (A on even
// sites, A^{-1} on odd sites) are staged into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier) when they fit; Sec. 3.3
// keeps each domain resident in a core's L2 for the same reason.  Then:
//
//   rho_Lambda += kappa * (hops from the neighbouring domains' last delta)
//                  [the inter-domain residual update of the previous
//                   half-sweep, pulled by the receiving domain: no atomics]
//   bhat_e = rho_e - D_eo A_oo^{-1} rho_o           (even-odd Schur RHS)
//   x_e = 0, r = bhat_e; nmr times:                  (MR on Dhat, Sec. 3.1 footnote)
//       p = Dhat r = A_ee r - D_eo A_oo^{-1} D_oe r   (hops leaving Lambda dropped)
//       alpha = <p, r> / <p, p>;  x_e += alpha r;  r -= alpha p
//   x_o = A_oo^{-1}(rho_o - D_oe x_e)
//   delta = (x_e, x_o);  psi_Lambda += delta;  rho_Lambda = (r, 0)
//
// D_eo = -kappa H_eo, D_oe = -kappa H_oe.  The odd half of the new domain
// residual is zero and the even half is the MR residual, so the residual on
// Lambda is set directly; the neighbours receive -D delta at the start of the
// next half-sweep.  Domain dot products: warp shuffles, then a fixed-order
// sum over warps in shared memory (deterministic).
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

// copy bytes (multiple of 16, both addresses 16-aligned) in chunks
__device__ __forceinline__ void bulk_g2s_chunked(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    const uint32_t kChunk = 32768;
    for (uint32_t off = 0; off < bytes; off += kChunk) {
        uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
        bulk_g2s((char *)dst + off, (const char *)src + off, n, bar);
    }
}

// ---------------------------------------------------------- kernel state

template <typename R, typename SL, typename SC, typename SS, typename SP>
struct SapArgs {
    Geom g;
    Field<SL> U;
    Field<SC> C;      // Schwarz clover: A on even sites, A^{-1} on odd sites
    Field<SS> rho;    // residual (read and written on the swept domains)
    Field<SS> delta;  // last correction of every domain
    Field<SP> psi;    // accumulated preconditioner output
    int64_t rstride;  // elements between right-hand sides (V*12)
    int64_t sstride;  // scale entries between right-hand sides (V)
    R kappa;
    int colour, nmr, nrhs, first_psi, gather, gather_only;
    int *err;
};

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

template <typename R, typename SL, typename SC>
__host__ __device__ constexpr size_t sap_smem_layout(int Vd, bool stl, bool stc)
{
    return (stl ? align128((size_t)36 * Vd * sizeof(typename SL::T2)) : 0) +
           (stc ? align128((size_t)36 * Vd * sizeof(typename SC::T2)) : 0) +
           ((stc && SC::kScaled) ? align128((size_t)Vd * 4) : 0) + 3 * align128((size_t)12 * (Vd / 2) * sizeof(cpx<R>)) +
           align128(128 * sizeof(R)) + align128(16);
}

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC>
struct SapBlock {
    const SapArgs<R, SL, SC, SS, SP> &a;
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

    // out = C(s) in : the Schwarz clover of this domain's site s, both blocks
    __device__ __forceinline__ void clover(int s, const cpx<R> *in, cpx<R> *out) const
    {
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            cpx<R> m[18];
            if (STC) {
                R sc = SC::kScaled ? (R)sCs[s] : (R)1;
#pragma unroll
                for (int k = 0; k < 18; k++) {
                    cpx<R> v = ld_s<R>(sC + (blk * 18 + k) * Vd + s);
                    m[k] = SC::kScaled ? sc * v : v;
                }
            } else {
                const typename SC::T2 *p = a.C.p + ((int64_t)d * 36 + blk * 18) * Vd + s;
                R sc = SC::kScaled ? (R)__ldg(a.C.scale + (int64_t)d * Vd + s) : (R)1;
#pragma unroll
                for (int k = 0; k < 18; k++) {
                    cpx<R> v = ld_c<R>(p + (int64_t)k * Vd);
                    m[k] = SC::kScaled ? sc * v : v;
                }
            }
            herm6_mul(m, in + 6 * blk, out + 6 * blk);
        }
    }

    // hops of site s from a shared-memory half-field (sites src_off..src_off+Vh-1),
    // dropping hops that leave the domain (Dirichlet boundary)
    template <int MU>
    __device__ __forceinline__ void inner_dir(int s, const uint16_t *nb, const cpx<R> *src, int src_off,
                                              cpx<R> *acc) const
    {
        cpx<R> u[9], x[12];
        uint16_t e = nb[2 * MU];
        if (!(e & kCross)) {
            int ns = (e & kSlotMask) - src_off;
#pragma unroll
            for (int k = 0; k < 12; k++) x[k] = src[k * Vh + ns];
            link(d, s, MU, u);
            hop<MU, +1>(u, x, acc);
        }
        e = nb[2 * MU + 1];
        if (!(e & kCross)) {
            int ns = e & kSlotMask;
#pragma unroll
            for (int k = 0; k < 12; k++) x[k] = src[k * Vh + ns - src_off];
            link(d, ns, MU, u);
            hop<MU, -1>(u, x, acc);
        }
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

    __device__ __forceinline__ void load_delta(int64_t rb, int64_t sb, int nd, int ns, cpx<R> *x) const
    {
        const typename SS::T2 *p = a.delta.p + rb + (int64_t)nd * 12 * Vd + ns;
        R sc = SS::kScaled ? (R)__ldg(a.delta.scale + sb + (int64_t)nd * Vd + ns) : (R)1;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            cpx<R> v = ld_c<R>(p + (int64_t)k * Vd);
            x[k] = SS::kScaled ? sc * v : v;
        }
    }

    // hops of site s from the neighbouring domains' delta (the hops that leave Lambda)
    template <int MU>
    __device__ __forceinline__ void outer_dir(int s, const uint16_t *nb, int64_t rb, int64_t sb, cpx<R> *acc) const
    {
        cpx<R> u[9], x[12];
        uint16_t e = nb[2 * MU];
        if (e & kCross) {
            int nd = __ldg(a.g.nbd + d * 8 + 2 * MU);
            load_delta(rb, sb, nd, e & kSlotMask, x);
            link(d, s, MU, u);
            hop<MU, +1>(u, x, acc);
        }
        e = nb[2 * MU + 1];
        if (e & kCross) {
            int nd = __ldg(a.g.nbd + d * 8 + 2 * MU + 1);
            int ns = e & kSlotMask;
            load_delta(rb, sb, nd, ns, x);
            link(nd, ns, MU, u);
            hop<MU, -1>(u, x, acc);
        }
    }

    __device__ __forceinline__ void outer_hops(int s, const uint16_t *nb, int64_t rb, int64_t sb, cpx<R> *acc) const
    {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
        outer_dir<0>(s, nb, rb, sb, acc);
        outer_dir<1>(s, nb, rb, sb, acc);
        outer_dir<2>(s, nb, rb, sb, acc);
        outer_dir<3>(s, nb, rb, sb, acc);
    }
};

template <typename R, typename S>
__device__ __forceinline__ void load_sp(const Field<S> &f, int64_t rb, int64_t sb, int d, int s, int Vd, cpx<R> *x)
{
    const typename S::T2 *p = f.p + rb + (int64_t)d * 12 * Vd + s;
    R sc = S::kScaled ? (R)f.scale[sb + (int64_t)d * Vd + s] : (R)1;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        cpx<R> v = ld_s<R>(p + (int64_t)k * Vd);
        x[k] = S::kScaled ? sc * v : v;
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
#pragma unroll
        for (int k = 0; k < 12; k++) st_c<R>(p + (int64_t)k * Vd, inv * x[k]);
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

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC>
__global__ void __launch_bounds__(256) k_sap(const SapArgs<R, SL, SC, SS, SP> a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_launch_dependents();
    const Geom &g = a.g;
    const int Vd = g.Vd, Vh = g.Vh;
    const int i = threadIdx.x;
    const int d = a.colour * g.Nd2 + blockIdx.x;
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
    R *sRed = (R *)ptr;           ptr += align128(128 * sizeof(R));
    uint64_t *bar = (uint64_t *)ptr;

    // stage the domain's links and clover blocks
    if (STL || STC) {
        if (i == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
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

    // neighbour slots of this thread's two sites, kept in registers
    uint16_t nbe[8], nbo[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        nbe[k] = __ldg(g.nbl + se * 8 + k);
        nbo[k] = __ldg(g.nbl + so * 8 + k);
    }

    SapBlock<R, SL, SC, SS, SP, STL, STC> B{a, d, Vd, Vh, sL, sC, sCs};
    const R kappa = a.kappa;
    const int nwarps = (Vh + 31) / 32;
    const bool full_warps = (Vh % 32) == 0;
    const int nphase = a.gather_only ? 0 : 3 + 2 * a.nmr;

    pdl_wait();  // the previous half-sweep's rho, delta and psi are visible from here on
    for (int rr = 0; rr < a.nrhs; rr++) {
        const int64_t rb = rr * a.rstride, sb = rr * a.sstride;

        if ((STL || STC) && rr == 0) {
            bool ok = mbar_wait_bounded(bar, 0, 1u << 22);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                // give the copies in flight a last bounded chance to land, then leave
                mbar_wait_bounded(bar, 0, 1u << 20);
                return;
            }
        }

        // residual of this domain plus the inflow from the other colour's
        // last corrections: rho += kappa * (hops that enter the domain)
        cpx<R> acc[12], v[12];
        for (int par = 0; par < 2; par++) {
            const int s = par ? so : se;
            load_sp<R, SS>(a.rho, rb, sb, d, s, Vd, v);
            if (a.gather) {
                uint16_t nb[8];
#pragma unroll
                for (int k = 0; k < 8; k++) nb[k] = par ? nbo[k] : nbe[k];
                B.outer_hops(s, nb, rb, sb, acc);
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = v[k] + kappa * acc[k];
            }
            if (a.gather_only) {
                store_sp<R, SS>(a.rho, rb, sb, d, s, Vd, v);
            } else {
                cpx<R> *dst = par ? sRo : sR;  // rho_e parks in sR until the setup phase
#pragma unroll
                for (int k = 0; k < 12; k++) dst[k * Vh + i] = v[k];
            }
        }
        if (a.gather_only) continue;

        cpx<R> r[12], x[12];
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
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    r[k] = sR[k * Vh + i] + kappa * acc[k];
                    sR[k * Vh + i] = a.nmr > 0 ? r[k] : x[k];
                }
                __syncthreads();
                continue;
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
                    if ((i & 31) == 0) {
                        sRed[(i >> 5) * 4 + 0] = pr_re;
                        sRed[(i >> 5) * 4 + 1] = pr_im;
                        sRed[(i >> 5) * 4 + 2] = pp;
                    }
                } else {
                    // partial warp (Vh < 32): per-thread partials, summed in order below
                    sRed[i * 3 + 0] = pr_re;
                    sRed[i * 3 + 1] = pr_im;
                    sRed[i * 3 + 2] = pp;
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
            } else if (type == PH_RECON_ODD) {
                // outputs: delta, psi, rho on this domain
                store_sp<R, SS>(a.delta, rb, sb, d, se, Vd, x);
                store_sp<R, SS>(a.delta, rb, sb, d, so, Vd, c);
                if (a.first_psi) {
                    store_sp<R, SP>(a.psi, rb, sb, d, se, Vd, x);
                    store_sp<R, SP>(a.psi, rb, sb, d, so, Vd, c);
                } else {
                    cpx<R> q[12];
                    load_sp<R, SP>(a.psi, rb, sb, d, se, Vd, q);
#pragma unroll
                    for (int k = 0; k < 12; k++) q[k] = q[k] + x[k];
                    store_sp<R, SP>(a.psi, rb, sb, d, se, Vd, q);
                    load_sp<R, SP>(a.psi, rb, sb, d, so, Vd, q);
#pragma unroll
                    for (int k = 0; k < 12; k++) q[k] = q[k] + c[k];
                    store_sp<R, SP>(a.psi, rb, sb, d, so, Vd, q);
                }
                store_sp<R, SS>(a.rho, rb, sb, d, se, Vd, r);
#pragma unroll
                for (int k = 0; k < 12; k++) c[k] = mk<R>(0, 0);
                store_sp<R, SS>(a.rho, rb, sb, d, so, Vd, c);
            } else {
                // setup-odd / mr-odd: t_o -> sT
#pragma unroll
                for (int k = 0; k < 12; k++) sT[k * Vh + i] = c[k];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Two threads per site pair.
//
// Thread h of a pair (lanes l and l + 16 of a warp) takes the hops in directions 2h and 2h+1
// (x, y for h = 0; z, t for h = 1) for both signs, then the pair exchanges
// partial sums with one shuffle so that thread h holds chirality h (spins
// 2h, 2h+1), applies clover block h and keeps that half of the MR state.
// Directions x and z, and y and t, differ in the spin algebra only by one
// sign and by whether the lower spins are swapped:
//   slot 0 (x or z):  a l = (-i l'_0, -i zeta l'_1)
//   slot 1 (y or t):  a l = (-zeta l'_0, l'_1)
// with zeta = +1 for h = 0 and -1 for h = 1, and l' the lower spins read in
// swapped order for h = 0.  The sign is a runtime factor inside an FMA and the
// swap is an address offset, so both threads of a warp run the same
// instructions: no divergence.  The lower-spin accumulator is kept in the
// same permuted order and put back in order at the exchange.

template <typename R>
struct PairHop {
    // acc_u[k] upper spin k, acc_l[k] lower spin pi(k) (permuted order)
    cpx<R> acc_u[2][3], acc_l[2][3];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc_u[k][c] = acc_l[k][c] = mk<R>(0, 0);
    }

    // one hop: x given as u[2][3] and l'[2][3] (lower spins permuted), U the link
    template <int SLOT, int SGN>
    __device__ __forceinline__ void hop(const cpx<R> (*u)[3], const cpx<R> (*l)[3], const cpx<R> *U, R zeta)
    {
        cpx<R> hh[2][3];
        const R s = (R)SGN;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (SLOT == 0) {
                // h0 = u0 + sgn i l'0 ; h1 = u1 + sgn zeta i l'1
                cpx<R> t0 = ti(l[0][c]);
                hh[0][c] = mk<R>(fma(s, t0.re, u[0][c].re), fma(s, t0.im, u[0][c].im));
                R sz = s * zeta;
                hh[1][c] = mk<R>(fma(-sz, l[1][c].im, u[1][c].re), fma(sz, l[1][c].re, u[1][c].im));
            } else {
                // h0 = u0 + sgn zeta l'0 ; h1 = u1 - sgn l'1
                R sz = s * zeta;
                hh[0][c] = mk<R>(fma(sz, l[0][c].re, u[0][c].re), fma(sz, l[0][c].im, u[0][c].im));
                hh[1][c] = mk<R>(fma(-s, l[1][c].re, u[1][c].re), fma(-s, l[1][c].im, u[1][c].im));
            }
        }
        cpx<R> w[2][3];
#pragma unroll
        for (int sp = 0; sp < 2; sp++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                cpx<R> t = mk<R>(0, 0);
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    if (SGN < 0) cfmac(t, U[b * 3 + a], hh[sp][b]);
                    else cfma(t, U[a * 3 + b], hh[sp][b]);
                }
                w[sp][a] = t;
            }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc_u[0][c] = acc_u[0][c] + w[0][c];
            acc_u[1][c] = acc_u[1][c] + w[1][c];
            if (SLOT == 0) {
                // acc'_0 += -sgn i w0 ; acc'_1 += -sgn zeta i w1
                cpx<R> t0 = ti(w[0][c]);
                acc_l[0][c] = mk<R>(fma(-s, t0.re, acc_l[0][c].re), fma(-s, t0.im, acc_l[0][c].im));
                R sz = s * zeta;
                acc_l[1][c] = mk<R>(fma(sz, w[1][c].im, acc_l[1][c].re), fma(-sz, w[1][c].re, acc_l[1][c].im));
            } else {
                // acc'_0 += sgn zeta w0 ; acc'_1 += -sgn w1
                R sz = s * zeta;
                acc_l[0][c] = mk<R>(fma(sz, w[0][c].re, acc_l[0][c].re), fma(sz, w[0][c].im, acc_l[0][c].im));
                acc_l[1][c] = mk<R>(fma(-s, w[1][c].re, acc_l[1][c].re), fma(-s, w[1][c].im, acc_l[1][c].im));
            }
        }
    }

    // partial sums of the pair -> chirality h of the total (6 complex, spin-major)
    __device__ __forceinline__ void exchange(int h, unsigned mask, cpx<R> *out) const
    {
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                // h = 0 keeps upper, sends lower in order (acc'_1, acc'_0);
                // h = 1 keeps lower (identity order), sends upper
                cpx<R> send = h ? acc_u[k][c] : acc_l[1 - k][c];
                cpx<R> keep = h ? acc_l[k][c] : acc_u[k][c];
                R rre = __shfl_xor_sync(mask, send.re, 16);
                R rim = __shfl_xor_sync(mask, send.im, 16);
                out[k * 3 + c] = mk<R>(keep.re + rre, keep.im + rim);
            }
    }
};

template <typename R, typename S>
__device__ __forceinline__ void load_half(const Field<S> &f, int64_t rb, int64_t sb, int d, int s, int Vd, int h,
                                          cpx<R> *x)
{
    const typename S::T2 *p = f.p + rb + ((int64_t)d * 12 + 6 * h) * Vd + s;
    R sc = S::kScaled ? (R)f.scale[sb + (int64_t)d * Vd + s] : (R)1;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        cpx<R> v = ld_s<R>(p + (int64_t)k * Vd);
        x[k] = S::kScaled ? sc * v : v;
    }
}

// both threads of the pair call this; 16-bit formats agree on one scale per site
template <typename R, typename S>
__device__ __forceinline__ void store_half(const Field<S> &f, int64_t rb, int64_t sb, int d, int s, int Vd, int h,
                                           unsigned mask, const cpx<R> *x)
{
    typename S::T2 *p = f.p + rb + ((int64_t)d * 12 + 6 * h) * Vd + s;
    if (S::kScaled) {
        R m = 0;
#pragma unroll
        for (int k = 0; k < 6; k++) m = fmax(m, fmax(fabs(x[k].re), fabs(x[k].im)));
        m = fmax(m, __shfl_xor_sync(mask, m, 16));
        float sc = (float)m;
        if (h == 0) f.scale[sb + (int64_t)d * Vd + s] = sc;
        R inv = m > 0 ? (R)1 / (R)sc : (R)0;
#pragma unroll
        for (int k = 0; k < 6; k++) st_c<R>(p + (int64_t)k * Vd, inv * x[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) st_c<R>(p + (int64_t)k * Vd, x[k]);
    }
}

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC>
struct PairBlock {
    const SapArgs<R, SL, SC, SS, SP> &a;
    int d, Vd, Vh, h;
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

    // out = block h of the Schwarz clover at site s times in (6 complex)
    __device__ __forceinline__ void clover(int s, const cpx<R> *in, cpx<R> *out) const
    {
        cpx<R> m[18];
        if (STC) {
            R sc = SC::kScaled ? (R)sCs[s] : (R)1;
#pragma unroll
            for (int k = 0; k < 18; k++) {
                cpx<R> v = ld_s<R>(sC + (h * 18 + k) * Vd + s);
                m[k] = SC::kScaled ? sc * v : v;
            }
        } else {
            const typename SC::T2 *p = a.C.p + ((int64_t)d * 36 + h * 18) * Vd + s;
            R sc = SC::kScaled ? (R)__ldg(a.C.scale + (int64_t)d * Vd + s) : (R)1;
#pragma unroll
            for (int k = 0; k < 18; k++) {
                cpx<R> v = ld_c<R>(p + (int64_t)k * Vd);
                m[k] = SC::kScaled ? sc * v : v;
            }
        }
        herm6_mul(m, in, out);
    }

    // spinor at slot ns of a shared half-field (sites off..off+Vh-1), lower spins permuted
    __device__ __forceinline__ void load_x_smem(const cpx<R> *src, int ns, cpx<R> (*u)[3], cpx<R> (*l)[3]) const
    {
        const int p0 = h ? 2 : 3, p1 = h ? 3 : 2;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            u[0][c] = src[(0 * 3 + c) * Vh + ns];
            u[1][c] = src[(1 * 3 + c) * Vh + ns];
            l[0][c] = src[(p0 * 3 + c) * Vh + ns];
            l[1][c] = src[(p1 * 3 + c) * Vh + ns];
        }
    }

    __device__ __forceinline__ void load_x_delta(int64_t rb, int64_t sb, int nd, int ns, cpx<R> (*u)[3],
                                                 cpx<R> (*l)[3]) const
    {
        const typename SS::T2 *p = a.delta.p + rb + (int64_t)nd * 12 * Vd + ns;
        R sc = SS::kScaled ? (R)__ldg(a.delta.scale + sb + (int64_t)nd * Vd + ns) : (R)1;
        const int p0 = h ? 2 : 3, p1 = h ? 3 : 2;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cpx<R> v;
            v = ld_c<R>(p + (int64_t)(0 * 3 + c) * Vd); u[0][c] = SS::kScaled ? sc * v : v;
            v = ld_c<R>(p + (int64_t)(1 * 3 + c) * Vd); u[1][c] = SS::kScaled ? sc * v : v;
            v = ld_c<R>(p + (int64_t)(p0 * 3 + c) * Vd); l[0][c] = SS::kScaled ? sc * v : v;
            v = ld_c<R>(p + (int64_t)(p1 * 3 + c) * Vd); l[1][c] = SS::kScaled ? sc * v : v;
        }
    }

    // this thread's two directions, hops inside the domain (Dirichlet)
    template <int SLOT>
    __device__ __forceinline__ void inner_slot(int s, const uint16_t *nb, const cpx<R> *src, int off, R zeta,
                                               PairHop<R> &H) const
    {
        const int mu = 2 * h + SLOT;
        cpx<R> u[2][3], l[2][3], U[9];
        uint16_t e = nb[2 * SLOT];
        if (!(e & kCross)) {
            load_x_smem(src, (e & kSlotMask) - off, u, l);
            link(d, s, mu, U);
            H.template hop<SLOT, +1>(u, l, U, zeta);
        }
        e = nb[2 * SLOT + 1];
        if (!(e & kCross)) {
            int ns = e & kSlotMask;
            load_x_smem(src, ns - off, u, l);
            link(d, ns, mu, U);
            H.template hop<SLOT, -1>(u, l, U, zeta);
        }
    }

    // hops entering from the neighbouring domains (their last delta)
    template <int SLOT>
    __device__ __forceinline__ void outer_slot(int s, const uint16_t *nb, int64_t rb, int64_t sb, R zeta,
                                               PairHop<R> &H) const
    {
        const int mu = 2 * h + SLOT;
        cpx<R> u[2][3], l[2][3], U[9];
        uint16_t e = nb[2 * SLOT];
        if (e & kCross) {
            int nd = __ldg(a.g.nbd + d * 8 + 2 * mu);
            load_x_delta(rb, sb, nd, e & kSlotMask, u, l);
            link(d, s, mu, U);
            H.template hop<SLOT, +1>(u, l, U, zeta);
        }
        e = nb[2 * SLOT + 1];
        if (e & kCross) {
            int nd = __ldg(a.g.nbd + d * 8 + 2 * mu + 1);
            int ns = e & kSlotMask;
            load_x_delta(rb, sb, nd, ns, u, l);
            link(nd, ns, mu, U);
            H.template hop<SLOT, -1>(u, l, U, zeta);
        }
    }
};

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC>
__global__ void __launch_bounds__(512, 1) k_sap_pair(const SapArgs<R, SL, SC, SS, SP> a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_launch_dependents();
    const Geom &g = a.g;
    const int Vd = g.Vd, Vh = g.Vh;
    // lanes l and l+16 of a warp form a pair: each half-warp reads one plane for
    // 16 consecutive sites, which keeps the 64-bit shared loads free of bank
    // conflicts (Vd must be a multiple of 32)
    const int t = threadIdx.x;
    const int i = (t >> 5) * 16 + (t & 15), h = (t >> 4) & 1;
    const int d = a.colour * g.Nd2 + blockIdx.x;
    const int se = i, so = Vh + i;
    const R zeta = h ? (R)-1 : (R)1;

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
    R *sRed = (R *)ptr;           ptr += align128(128 * sizeof(R));
    uint64_t *bar = (uint64_t *)ptr;

    if (STL || STC) {
        if (t == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (t == 0) {
            uint32_t lb = STL ? (uint32_t)(36 * Vd * sizeof(typename SL::T2)) : 0;
            uint32_t cb = STC ? (uint32_t)(36 * Vd * sizeof(typename SC::T2)) : 0;
            uint32_t sb = (STC && SC::kScaled) ? (uint32_t)(Vd * 4) : 0;
            mbar_arrive_expect_tx(bar, lb + cb + sb);
            if (STL) bulk_g2s_chunked(sL, a.U.p + (int64_t)d * 36 * Vd, lb, bar);
            if (STC) bulk_g2s_chunked(sC, a.C.p + (int64_t)d * 36 * Vd, cb, bar);
            if (STC && SC::kScaled) bulk_g2s_chunked(sCs, a.C.scale + (int64_t)d * Vd, sb, bar);
        }
    }

    // this thread's neighbour entries: directions 2h, 2h+1, both signs, for both sites
    uint16_t nbe[4], nbo[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        nbe[k] = __ldg(g.nbl + se * 8 + 4 * h + k);
        nbo[k] = __ldg(g.nbl + so * 8 + 4 * h + k);
    }

    PairBlock<R, SL, SC, SS, SP, STL, STC> B{a, d, Vd, Vh, h, sL, sC, sCs};
    const R kappa = a.kappa;
    const int nthreads = Vd;
    const int nwarps = (nthreads + 31) / 32;
    const bool full_warps = (nthreads % 32) == 0;
    const unsigned mask = 0xffffffffu;
    const int nphase = a.gather_only ? 0 : 3 + 2 * a.nmr;

    pdl_wait();  // the previous half-sweep's rho, delta and psi are visible from here on
    for (int rr = 0; rr < a.nrhs; rr++) {
        const int64_t rb = rr * a.rstride, sb = rr * a.sstride;

        if ((STL || STC) && rr == 0) {
            bool ok = mbar_wait_bounded(bar, 0, 1u << 22);
            if (!ok) atomicOr(a.err, kErrMbarTimeout);
            if (__syncthreads_or(!ok)) {
                mbar_wait_bounded(bar, 0, 1u << 20);
                return;
            }
        }

        PairHop<R> H;
        cpx<R> v[6];
        for (int par = 0; par < 2; par++) {
            const int s = par ? so : se;
            load_half<R, SS>(a.rho, rb, sb, d, s, Vd, h, v);
            if (a.gather) {
                uint16_t nb[4];
#pragma unroll
                for (int k = 0; k < 4; k++) nb[k] = par ? nbo[k] : nbe[k];
                H.zero();
                B.template outer_slot<0>(s, nb, rb, sb, zeta, H);
                B.template outer_slot<1>(s, nb, rb, sb, zeta, H);
                cpx<R> in[6];
                H.exchange(h, mask, in);
#pragma unroll
                for (int k = 0; k < 6; k++) v[k] = v[k] + kappa * in[k];
            }
            if (a.gather_only) {
                store_half<R, SS>(a.rho, rb, sb, d, s, Vd, h, mask, v);
            } else {
                cpx<R> *dst = par ? sRo : sR;
#pragma unroll
                for (int k = 0; k < 6; k++) dst[(6 * h + k) * Vh + i] = v[k];
            }
        }
        if (a.gather_only) continue;

        cpx<R> r[6], x[6];
#pragma unroll
        for (int k = 0; k < 6; k++) x[k] = mk<R>(0, 0);

        for (int ph = 0; ph < nphase; ph++) {
            const int type = ph == 0 ? PH_SETUP_ODD
                             : ph == 1 ? PH_SETUP_EVEN
                             : ph == nphase - 1 ? PH_RECON_ODD
                             : ((ph & 1) ? PH_MR_EVEN : PH_MR_ODD);
            const int par = (type == PH_SETUP_EVEN || type == PH_MR_EVEN) ? 0 : 1;
            const int s = par ? so : se;

            cpx<R> acc[6];
            if (type != PH_SETUP_ODD) {
                uint16_t nb[4];
#pragma unroll
                for (int k = 0; k < 4; k++) nb[k] = par ? nbo[k] : nbe[k];
                const cpx<R> *src = par ? sR : sT;
                const int off = par ? 0 : Vh;
                H.zero();
                B.template inner_slot<0>(s, nb, src, off, zeta, H);
                B.template inner_slot<1>(s, nb, src, off, zeta, H);
                H.exchange(h, mask, acc);
            } else {
#pragma unroll
                for (int k = 0; k < 6; k++) acc[k] = mk<R>(0, 0);
            }

            if (type == PH_SETUP_EVEN) {
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    r[k] = sR[(6 * h + k) * Vh + i] + kappa * acc[k];
                    sR[(6 * h + k) * Vh + i] = a.nmr > 0 ? r[k] : x[k];
                }
                __syncthreads();
                continue;
            }
#pragma unroll
            for (int k = 0; k < 6; k++) {
                cpx<R> own = type == PH_MR_EVEN ? r[k]
                             : (type == PH_MR_ODD ? mk<R>(0, 0) : sRo[(6 * h + k) * Vh + i]);
                R ka = type == PH_MR_EVEN || type == PH_SETUP_ODD ? (R)0 : (type == PH_MR_ODD ? -kappa : kappa);
                v[k] = own + ka * acc[k];
            }
            cpx<R> c[6];
            B.clover(s, v, c);

            if (type == PH_MR_EVEN) {
                R pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
                for (int k = 0; k < 6; k++) {
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
                    if ((t & 31) == 0) {
                        sRed[(t >> 5) * 4 + 0] = pr_re;
                        sRed[(t >> 5) * 4 + 1] = pr_im;
                        sRed[(t >> 5) * 4 + 2] = pp;
                    }
                } else {
                    sRed[t * 3 + 0] = pr_re;
                    sRed[t * 3 + 1] = pr_im;
                    sRed[t * 3 + 2] = pp;
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
                    for (int w = 0; w < nthreads; w++) {
                        tr += sRed[w * 3 + 0];
                        ti_ += sRed[w * 3 + 1];
                        tp += sRed[w * 3 + 2];
                    }
                }
                cpx<R> alpha = tp > (R)0 ? mk<R>(tr / tp, ti_ / tp) : mk<R>(0, 0);
                const bool last = ph == nphase - 2;
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    cfma(x[k], alpha, r[k]);
                    r[k] = r[k] - alpha * c[k];
                    sR[(6 * h + k) * Vh + i] = last ? x[k] : r[k];
                }
            } else if (type == PH_RECON_ODD) {
                store_half<R, SS>(a.delta, rb, sb, d, se, Vd, h, mask, x);
                store_half<R, SS>(a.delta, rb, sb, d, so, Vd, h, mask, c);
                if (a.first_psi) {
                    store_half<R, SP>(a.psi, rb, sb, d, se, Vd, h, mask, x);
                    store_half<R, SP>(a.psi, rb, sb, d, so, Vd, h, mask, c);
                } else {
                    cpx<R> q[6];
                    load_half<R, SP>(a.psi, rb, sb, d, se, Vd, h, q);
#pragma unroll
                    for (int k = 0; k < 6; k++) q[k] = q[k] + x[k];
                    store_half<R, SP>(a.psi, rb, sb, d, se, Vd, h, mask, q);
                    load_half<R, SP>(a.psi, rb, sb, d, so, Vd, h, q);
#pragma unroll
                    for (int k = 0; k < 6; k++) q[k] = q[k] + c[k];
                    store_half<R, SP>(a.psi, rb, sb, d, so, Vd, h, mask, q);
                }
                store_half<R, SS>(a.rho, rb, sb, d, se, Vd, h, mask, r);
#pragma unroll
                for (int k = 0; k < 6; k++) c[k] = mk<R>(0, 0);
                store_half<R, SS>(a.rho, rb, sb, d, so, Vd, h, mask, c);
            } else {
#pragma unroll
                for (int k = 0; k < 6; k++) sT[(6 * h + k) * Vh + i] = c[k];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- launch

template <typename R, typename SL, typename SC, typename SS, typename SP, bool STL, bool STC, bool PAIR>
static qdd_status run_sap(Gauge *g, const SapArgs<R, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl, bool timed)
{
    const HostGeom &hg = g->hg;
    size_t smem = sap_smem_layout<R, SL, SC>(hg.Vd, STL, STC);
    auto kern = [] {
        if constexpr (PAIR) return k_sap_pair<R, SL, SC, SS, SP, STL, STC>;
        else return k_sap<R, SL, SC, SS, SP, STL, STC>;
    }();
    static thread_local size_t configured = 0;
    if (configured < smem) {
        QDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(hg.Nd2);
    cfg.blockDim = dim3(PAIR ? hg.Vd : hg.Vh);
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

template <typename R, typename SL, typename SC, typename SS, typename SP, bool PAIR>
static qdd_status dispatch_staging_v(Gauge *g, const SapArgs<R, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl,
                                     bool timed)
{
    const int Vd = g->hg.Vd;
    const size_t lim = smem_limit();
    if (sap_smem_layout<R, SL, SC>(Vd, true, true) <= lim)
        return run_sap<R, SL, SC, SS, SP, true, true, PAIR>(g, a, s, pdl, timed);
    if (sap_smem_layout<R, SL, SC>(Vd, true, false) <= lim)
        return run_sap<R, SL, SC, SS, SP, true, false, PAIR>(g, a, s, pdl, timed);
    if (sap_smem_layout<R, SL, SC>(Vd, false, false) <= lim)
        return run_sap<R, SL, SC, SS, SP, false, false, PAIR>(g, a, s, pdl, timed);
    set_error("domain of %d sites does not fit in shared memory", Vd);
    return QDD_EINVAL;
}

// Kernel variant: one thread per even/odd site pair, or two (FP32 arithmetic
// and domains of a multiple of 32 sites).  The gauge field's sap_variant
// selects (0 = automatic = one thread per pair, measured faster on GB300:
// the pair form halves the registers but issues 30% more instructions).
template <typename R, typename SL, typename SC, typename SS, typename SP>
static qdd_status dispatch_staging(Gauge *g, const SapArgs<R, SL, SC, SS, SP> &a, cudaStream_t s, bool pdl,
                                   bool timed)
{
    if constexpr (std::is_same<R, float>::value) {
        if (g->sap_variant == 2 && g->hg.Vd % 32 == 0)
            return dispatch_staging_v<R, SL, SC, SS, SP, true>(g, a, s, pdl, timed);
    }
    return dispatch_staging_v<R, SL, SC, SS, SP, false>(g, a, s, pdl, timed);
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
                                bool timed)
{
    QDD_TRY(ensure_copy(g, prec, s));
    const int64_t rs = (int64_t)g->hg.V * 12, ss = g->hg.V;
    PrecCopy &c = g->copies[prec];
    switch (prec) {
    case QDD_PREC_F64: {
        SapArgs<double, StF64, StF64, StF64, StF64> a{
            g->geom, {g->links64.as<double2>(), nullptr}, {g->sclov64.as<double2>(), nullptr},
            {(double2 *)b.rho, nullptr}, {(double2 *)b.delta, nullptr}, {(double2 *)b.psi, nullptr},
            rs, ss, g->kappa, colour, nmr, nrhs, first_psi, gather, gather_only, d_err};
        return dispatch_staging(g, a, s, pdl, timed);
    }
    case QDD_PREC_F32: {
        SapArgs<float, StF32, StF32, StF32, StF32> a{
            g->geom, {c.links.as<float2>(), nullptr}, {c.sclov.as<float2>(), nullptr},
            {(float2 *)b.rho, nullptr}, {(float2 *)b.delta, nullptr}, {(float2 *)b.psi, nullptr},
            rs, ss, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, gather_only, d_err};
        return dispatch_staging(g, a, s, pdl, timed);
    }
    case QDD_PREC_F16S: {
        SapArgs<float, StF16, StF16, StF16, StF32> a{
            g->geom, {c.links.as<__half2>(), nullptr}, {c.sclov.as<__half2>(), c.sclov_s.as<float>()},
            {(__half2 *)b.rho, b.rho_s}, {(__half2 *)b.delta, b.delta_s}, {(float2 *)b.psi, nullptr},
            rs, ss, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, gather_only, d_err};
        return dispatch_staging(g, a, s, pdl, timed);
    }
    case QDD_PREC_H16: {
        PrecCopy &h = g->copies[QDD_PREC_F16S];
        SapArgs<float, StF16, StF16, StF32, StF32> a{
            g->geom, {h.links.as<__half2>(), nullptr}, {h.sclov.as<__half2>(), h.sclov_s.as<float>()},
            {(float2 *)b.rho, nullptr}, {(float2 *)b.delta, nullptr}, {(float2 *)b.psi, nullptr},
            rs, ss, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, gather_only, d_err};
        return dispatch_staging(g, a, s, pdl, timed);
    }
    case QDD_PREC_BF16S: {
        SapArgs<float, StBF16, StBF16, StBF16, StF32> a{
            g->geom, {c.links.as<__nv_bfloat162>(), nullptr}, {c.sclov.as<__nv_bfloat162>(), c.sclov_s.as<float>()},
            {(__nv_bfloat162 *)b.rho, b.rho_s}, {(__nv_bfloat162 *)b.delta, b.delta_s}, {(float2 *)b.psi, nullptr},
            rs, ss, (float)g->kappa, colour, nmr, nrhs, first_psi, gather, gather_only, d_err};
        return dispatch_staging(g, a, s, pdl, timed);
    }
    default: break;
    }
    set_error("invalid preconditioner precision %d", (int)prec);
    return QDD_EINVAL;
}

}  // namespace qdd
