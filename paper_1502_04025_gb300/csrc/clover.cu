// Clover term of the Wilson-clover operator (arXiv:1502.04025, Sec. 3.1
// names the operator; Sec. 3.6 counts 1848 flop per site for it).
//
//   A(n) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(n),
//   F_{mu nu} = traceless part of (Q_{mu nu} - Q_{mu nu}^+)/8, Q the four-leaf
//   clover of plaquettes at n in the (mu, nu) plane.
// In the chiral basis sigma_{mu nu} is block diagonal: A is two Hermitian 6x6
// blocks (spins {0,1} and {2,3}), each  1 + i kappa c_sw sum_k sigma_k (x) G_k,
// with G_k = B_k +- E_k, B = (-F_yz, F_xz, -F_xy), E_k = F_kt (+ for the
// upper block, - for the lower).  The even-odd domain solver also needs the
// inverse blocks on odd sites (the Schwarz form keeps A on even sites and
// A^{-1} on odd sites).  Built in FP64 once per (gauge, c_sw, kappa).
#include "internal.h"

namespace qdd {

typedef cpx<double> zd;

struct M3 {
    zd m[9];
};

__device__ __forceinline__ M3 load_link(const Geom &g, const double2 *U, int gi, int mu)
{
    M3 r;
    int d, s;
    split_index(g, gi, d, s);
    const double2 *p = U + ((int64_t)d * 36 + mu * 9) * g.Vd + s;
    for (int k = 0; k < 9; k++) {
        double2 v = __ldg(p + (int64_t)k * g.Vd);
        r.m[k] = mk(v.x, v.y);
    }
    return r;
}

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            zd acc = mk(0.0, 0.0);
            for (int k = 0; k < 3; k++) cfma(acc, a.m[i * 3 + k], b.m[k * 3 + j]);
            r.m[i * 3 + j] = acc;
        }
    return r;
}

__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.m[i * 3 + j] = conj(a.m[j * 3 + i]);
    return r;
}

__device__ __forceinline__ int nbr(const Geom &g, int gi, int k)
{
    int d, s;
    split_index(g, gi, d, s);
    return neighbour(g, d, s, k);
}

// F_{mu nu} at gi
__device__ M3 field_strength(const Geom &g, const double2 *U, int gi, int mu, int nu)
{
    int n_pm = nbr(g, gi, 2 * mu), n_mm = nbr(g, gi, 2 * mu + 1);
    int n_pn = nbr(g, gi, 2 * nu), n_mn = nbr(g, gi, 2 * nu + 1);
    int n_mm_pn = nbr(g, n_mm, 2 * nu), n_mm_mn = nbr(g, n_mm, 2 * nu + 1);
    int n_pm_mn = nbr(g, n_pm, 2 * nu + 1);
    M3 Umu = load_link(g, U, gi, mu), Unu = load_link(g, U, gi, nu);
    // leaf 1: n -> n+mu -> n+mu+nu -> n+nu -> n
    M3 q = mul(mul(Umu, load_link(g, U, n_pm, nu)), mul(dag(load_link(g, U, n_pn, mu)), dag(Unu)));
    // leaf 2: n -> n+nu -> n+nu-mu -> n-mu -> n
    M3 l = mul(mul(Unu, dag(load_link(g, U, n_mm_pn, mu))),
               mul(dag(load_link(g, U, n_mm, nu)), load_link(g, U, n_mm, mu)));
    for (int k = 0; k < 9; k++) q.m[k] = q.m[k] + l.m[k];
    // leaf 3: n -> n-mu -> n-mu-nu -> n-nu -> n
    l = mul(mul(dag(load_link(g, U, n_mm, mu)), dag(load_link(g, U, n_mm_mn, nu))),
            mul(load_link(g, U, n_mm_mn, mu), load_link(g, U, n_mn, nu)));
    for (int k = 0; k < 9; k++) q.m[k] = q.m[k] + l.m[k];
    // leaf 4: n -> n-nu -> n-nu+mu -> n+mu -> n
    l = mul(mul(dag(load_link(g, U, n_mn, nu)), load_link(g, U, n_mn, mu)),
            mul(load_link(g, U, n_pm_mn, nu), dag(Umu)));
    for (int k = 0; k < 9; k++) q.m[k] = q.m[k] + l.m[k];
    M3 F;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) F.m[a * 3 + b] = 0.125 * (q.m[a * 3 + b] - conj(q.m[b * 3 + a]));
    zd tr = (1.0 / 3.0) * (F.m[0] + F.m[4] + F.m[8]);
    F.m[0] = F.m[0] - tr;
    F.m[4] = F.m[4] - tr;
    F.m[8] = F.m[8] - tr;
    return F;
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting
__device__ bool invert6(zd *M /* 36, overwritten */, zd *inv /* 36 */)
{
    for (int i = 0; i < 36; i++) inv[i] = mk(0.0, 0.0);
    for (int i = 0; i < 6; i++) inv[i * 6 + i] = mk(1.0, 0.0);
    for (int c = 0; c < 6; c++) {
        int piv = c;
        double best = M[c * 6 + c].re * M[c * 6 + c].re + M[c * 6 + c].im * M[c * 6 + c].im;
        for (int r = c + 1; r < 6; r++) {
            double v = M[r * 6 + c].re * M[r * 6 + c].re + M[r * 6 + c].im * M[r * 6 + c].im;
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < 6; j++) {
                zd t = M[c * 6 + j]; M[c * 6 + j] = M[piv * 6 + j]; M[piv * 6 + j] = t;
                t = inv[c * 6 + j]; inv[c * 6 + j] = inv[piv * 6 + j]; inv[piv * 6 + j] = t;
            }
        zd p = M[c * 6 + c];
        zd pinv = (1.0 / best) * conj(p);
        for (int j = 0; j < 6; j++) {
            M[c * 6 + j] = M[c * 6 + j] * pinv;
            inv[c * 6 + j] = inv[c * 6 + j] * pinv;
        }
        for (int r = 0; r < 6; r++) {
            if (r == c) continue;
            zd f = M[r * 6 + c];
            for (int j = 0; j < 6; j++) {
                M[r * 6 + j] = M[r * 6 + j] - f * M[c * 6 + j];
                inv[r * 6 + j] = inv[r * 6 + j] - f * inv[c * 6 + j];
            }
        }
    }
    return true;
}

__device__ __forceinline__ void pack_herm6(const zd *M, double2 *dst, int64_t stride)
{
    dst[0] = make_double2(M[0].re, M[7].re);
    dst[stride] = make_double2(M[14].re, M[21].re);
    dst[2 * stride] = make_double2(M[28].re, M[35].re);
    int k = 3;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            // symmetrise the rounding of the two triangles
            zd v = 0.5 * (M[i * 6 + j] + conj(M[j * 6 + i]));
            dst[k * stride] = make_double2(v.re, v.im);
            k++;
        }
}

__global__ void k_clover_build(Geom g, const double2 *U, double csw, double kappa, double2 *A, double2 *S,
                               int *singular)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.V) return;
    int d, s;
    split_index(g, gi, d, s);
    // F in the order (xy, xz, xt, yz, yt, zt)
    M3 Fxy = field_strength(g, U, gi, 0, 1), Fxz = field_strength(g, U, gi, 0, 2);
    M3 Fxt = field_strength(g, U, gi, 0, 3), Fyz = field_strength(g, U, gi, 1, 2);
    M3 Fyt = field_strength(g, U, gi, 1, 3), Fzt = field_strength(g, U, gi, 2, 3);
    bool odd = s >= g.Vh;
    const double kc = kappa * csw;
    for (int ch = 0; ch < 2; ch++) {
        double se = ch == 0 ? 1.0 : -1.0;
        zd G1[9], G2[9], G3[9];
        for (int k = 0; k < 9; k++) {
            G1[k] = (-1.0) * Fyz.m[k] + se * Fxt.m[k];
            G2[k] = Fxz.m[k] + se * Fyt.m[k];
            G3[k] = (-1.0) * Fxy.m[k] + se * Fzt.m[k];
        }
        zd M[36];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                zd g3 = G3[a * 3 + b];
                zd c01 = G1[a * 3 + b] - ti(G2[a * 3 + b]);  // (sigma_1 G1 + sigma_2 G2)_{01}
                zd c10 = G1[a * 3 + b] + ti(G2[a * 3 + b]);  // (...)_{10}
                // M = 1 + i kappa c_sw (...)
                M[(0 * 3 + a) * 6 + 0 * 3 + b] = kc * ti(g3);
                M[(1 * 3 + a) * 6 + 1 * 3 + b] = kc * ti(-g3);
                M[(0 * 3 + a) * 6 + 1 * 3 + b] = kc * ti(c01);
                M[(1 * 3 + a) * 6 + 0 * 3 + b] = kc * ti(c10);
            }
        for (int i = 0; i < 6; i++) M[i * 6 + i].re += 1.0;
        const int64_t base = ((int64_t)d * 36 + ch * 18) * g.Vd + s;
        pack_herm6(M, A + base, g.Vd);
        if (!odd) {
            pack_herm6(M, S + base, g.Vd);
        } else {
            zd inv[36];
            if (!invert6(M, inv)) {
                atomicAdd(singular, 1);
                for (int i = 0; i < 36; i++) inv[i] = mk(0.0, 0.0);
            }
            pack_herm6(inv, S + base, g.Vd);
        }
    }
}

qdd_status launch_clover_build(Gauge *g, double csw, double kappa, int *d_singular, cudaStream_t s)
{
    LaunchScope ls(g->ctx->timer, K_OTHER, s);
    k_clover_build<<<(g->hg.V + 127) / 128, 128, 0, s>>>(g->geom, g->links64.as<double2>(), csw, kappa,
                                                        g->clov64.as<double2>(), g->sclov64.as<double2>(),
                                                        d_singular);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

}  // namespace qdd
