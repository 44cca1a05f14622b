// A lattice sharded in the time direction over ranks (arXiv:1502.04025,
// Sec. 3.6: the lattice is distributed over processors and the domain
// boundaries are exchanged).  Each rank owns a slab of whole domains and
// computes with its local lattice wrapped periodically in t, so that every
// kernel of the single-GPU path runs unchanged; what the wrap gets wrong is
// confined to the slab's two boundary planes and is exchanged here.
//
//   Schwarz half-sweep   A domain pushes each hop of its correction that
//                        leaves it into a face slot of the receiving domain,
//                        computed from the pushing side's data alone (its
//                        correction and its own link).  Across the wrap, the
//                        last t-block's pushes land in the first t-block's
//                        "from below" slots and the first t-block's in the
//                        last's "from above" slots: exactly what the ranks
//                        above and below need.  A cyclic shift of those two
//                        slot regions after every half-sweep makes every
//                        slot hold what a single lattice would (bit for bit:
//                        one writer per slot, summed by the receiver in a
//                        fixed order).
//   operator D           The hops across the wrap at planes 0 and lt-1 took
//                        the rank's own far plane.  Each rank packs, for its
//                        last plane, the backward hop it sends up
//                        (U_t^+ (1 + gamma_t) psi, projected) and, for its
//                        first plane, the forward hop's projected spinor
//                        ((1 - gamma_t) psi); after a cyclic shift the
//                        boundary planes add kappa times (wrapped - received).
//   clover term          The four-leaf clover of a boundary plane needs links
//                        one plane beyond it: the clover is built on an
//                        extended lattice with one domain block of halo on
//                        each side and the owned sites take theirs.
//   FGMRES               Dot products and norms are summed over the ranks.
// The exchanges follow the overlap order of Sec. 3.6: a half-sweep runs the
// first and last t-block's domains first and the interior second, and their
// face slots move on a side stream (through page-locked host memory and the
// caller's shift hook) while the interior computes; the operator's boundary
// planes are packed and shifted while the operator runs.
#include <cstring>

#include "internal.h"

namespace qdd {

Slab::~Slab()
{
    if (side) cudaStreamSynchronize(side);
    for (void *h : {host_face, host_op, host_red})
        if (h) cudaFreeHost(h);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (side) cudaStreamDestroy(side);
    if (ext) qdd_destroy_gauge(ext);
}

void slab_regions(const HostGeom &hg, int colour, int out[6])
{
    const int recv = 1 - (colour & 1);  // colour of the receiving domains
    const int half = hg.nb[0] * hg.nb[1] * hg.nb[2] / 2;  // domains of one colour in one t-block
    // first t-block (slots 0 .. half-1 of a colour): the slots fed from below (direction 7)
    out[0] = recv * hg.Nd2;
    out[1] = half;
    out[2] = 7;
    // last t-block (the last half slots of a colour): the slots fed from above (direction 6)
    out[3] = recv * hg.Nd2 + hg.Nd2 - half;
    out[4] = half;
    out[5] = 6;
}

// grow a page-locked staging buffer (after the side stream's copies from it)
static qdd_status ensure_host(Slab &sl, void *&h, size_t &have, size_t bytes)
{
    if (h && have >= bytes) return QDD_OK;
    QDD_CUDA(cudaStreamSynchronize(sl.side));
    if (h) cudaFreeHost(h);
    h = nullptr;
    have = 0;
    QDD_CUDA(cudaMallocHost(&h, bytes));
    have = bytes;
    return QDD_OK;
}

static qdd_status shift(Slab &sl, const void *to_up, void *from_dn, const void *to_dn, void *from_up, size_t bytes)
{
    if (sl.comm.shift(sl.comm.user, to_up, from_dn, to_dn, from_up, bytes) != 0) {
        set_error("the shift hook of rank %d failed", sl.comm.rank);
        return QDD_ECOMM;
    }
    return QDD_OK;
}

qdd_status slab_allreduce(Gauge *g, double *host, size_t n)
{
    if (!g->slab || n == 0) return QDD_OK;
    Slab &sl = *g->slab;
    if (sl.comm.allreduce_sum(sl.comm.user, host, n) != 0) {
        set_error("the allreduce hook of rank %d failed", sl.comm.rank);
        return QDD_ECOMM;
    }
    return QDD_OK;
}

qdd_status slab_allreduce_dev(Gauge *g, double2 *dev, int n, cudaStream_t s)
{
    if (!g->slab || n <= 0) return QDD_OK;
    Slab &sl = *g->slab;
    const size_t bytes = (size_t)n * sizeof(double2);
    QDD_TRY(ensure_host(sl, sl.host_red, sl.red_bytes, bytes));
    QDD_CUDA(cudaMemcpyAsync(sl.host_red, dev, bytes, cudaMemcpyDeviceToHost, s));
    QDD_CUDA(cudaStreamSynchronize(s));
    QDD_TRY(slab_allreduce(g, (double *)sl.host_red, 2 * (size_t)n));
    QDD_CUDA(cudaMemcpyAsync(dev, sl.host_red, bytes, cudaMemcpyHostToDevice, s));
    // the staging buffer is reused by the next sum: let the copy finish
    QDD_CUDA(cudaStreamSynchronize(s));
    return QDD_OK;
}

qdd_status slab_sap_halfsweep(Gauge *g, qdd_prec prec, const SapBuffers &b, int colour, int nmr, int nrhs,
                              int first_psi, int gather, int *d_err, cudaStream_t s, bool exchange)
{
    Slab &sl = *g->slab;
    const HostGeom &hg = g->hg;
    // boundary t-blocks first
    QDD_TRY(launch_sap_halfsweep(g, prec, b, colour, nmr, nrhs, first_psi, gather, 0, d_err, s, false, false, 1));
    if (exchange) QDD_CUDA(cudaEventRecord(sl.ev_in, s));
    QDD_TRY(launch_sap_halfsweep(g, prec, b, colour, nmr, nrhs, first_psi, gather, 0, d_err, s, false, false, 2));
    if (!exchange) return QDD_OK;
    // meanwhile: the slots the boundary domains pushed across the slab
    // boundaries (regions that no interior domain writes or reads)
    const size_t esz = prec == QDD_PREC_F64 ? sizeof(double2) : sizeof(float2);
    int r[6];
    slab_regions(hg, colour, r);
    const size_t count = (size_t)hg.Vd / hg.dom[3];  // slots of a t face
    const size_t width = count * esz, pitch = (size_t)hg.nf * esz;
    const size_t rows = (size_t)r[1] * 6;
    const size_t rb = rows * width;                  // one region of one right-hand side
    const size_t fstride = (size_t)hg.Nd * 6 * hg.nf * esz;
    const size_t tot = rb * nrhs;
    QDD_TRY(ensure_host(sl, sl.host_face, sl.face_bytes, 4 * tot));
    char *h = (char *)sl.host_face;
    char *up = h, *dn = h + tot, *from_dn = h + 2 * tot, *from_up = h + 3 * tot;
    char *f = (char *)b.face;
    QDD_CUDA(cudaStreamWaitEvent(sl.side, sl.ev_in, 0));
    for (int k = 0; k < nrhs; k++) {
        const char *ru = f + k * fstride + ((size_t)r[0] * 6 * hg.nf + hg.foff[r[2]]) * esz;
        const char *rd = f + k * fstride + ((size_t)r[3] * 6 * hg.nf + hg.foff[r[5]]) * esz;
        QDD_CUDA(cudaMemcpy2DAsync(up + k * rb, width, ru, pitch, width, rows, cudaMemcpyDeviceToHost, sl.side));
        QDD_CUDA(cudaMemcpy2DAsync(dn + k * rb, width, rd, pitch, width, rows, cudaMemcpyDeviceToHost, sl.side));
    }
    QDD_CUDA(cudaStreamSynchronize(sl.side));  // the interior may still be running
    QDD_TRY(shift(sl, up, from_dn, dn, from_up, tot));
    for (int k = 0; k < nrhs; k++) {
        char *ru = f + k * fstride + ((size_t)r[0] * 6 * hg.nf + hg.foff[r[2]]) * esz;
        char *rd = f + k * fstride + ((size_t)r[3] * 6 * hg.nf + hg.foff[r[5]]) * esz;
        QDD_CUDA(cudaMemcpy2DAsync(ru, pitch, from_dn + k * rb, width, width, rows, cudaMemcpyHostToDevice, sl.side));
        QDD_CUDA(cudaMemcpy2DAsync(rd, pitch, from_up + k * rb, width, width, rows, cudaMemcpyHostToDevice, sl.side));
    }
    QDD_CUDA(cudaEventRecord(sl.ev_out, sl.side));
    QDD_CUDA(cudaStreamWaitEvent(s, sl.ev_out, 0));
    return QDD_OK;
}

// --------------------------------------------------------- operator planes

// element offset of component k of boundary site j on plane p (0: t = 0,
// 1: t = lt-1): the internal layout from the table, else the host layout
struct PlaneAddr {
    const int64_t *base;  // [2][Ls] or NULL for the host layout
    int64_t cstride;      // Vd (internal) or 1 (host layout)
    int Ls, lt;
    __device__ __forceinline__ int64_t at(int p, int j) const
    {
        return base ? __ldg(base + (int64_t)p * Ls + j) : ((int64_t)j + (p ? (int64_t)(lt - 1) * Ls : 0)) * 12;
    }
};

template <typename T2>
__device__ __forceinline__ cpx<double> ld_any(const T2 *p)
{
    T2 v = *p;
    return mk<double>((double)v.x, (double)v.y);
}

// own[0]: U_t^+ (1 + gamma_t) x projected at plane lt-1 (the backward hop sent up);
// own[1]: (1 - gamma_t) x projected at plane 0 (the forward hop sent down)
template <typename T2>
__global__ void __launch_bounds__(128) k_slab_pack(const T2 *x, PlaneAddr pa, int64_t fstride, const double2 *U,
                                                   const int64_t *last_link, int64_t lstride, int nrhs,
                                                   double2 *own_b, double2 *own_f)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (j >= pa.Ls || r >= nrhs) return;
    cpx<double> v[12], h[6], w[6], u[9];
    int64_t a = pa.at(1, j) + r * fstride;
    for (int k = 0; k < 12; k++) v[k] = ld_any(x + a + k * pa.cstride);
    project<3, -1>(v, h);
    const int64_t lb = __ldg(last_link + j);
    for (int k = 0; k < 9; k++) {
        double2 e = __ldg(U + lb + k * lstride);
        u[k] = mk(e.x, e.y);
    }
    su3_mul_half<true>(u, h, w);
    double2 *ob = own_b + ((int64_t)r * pa.Ls + j) * 6;
    for (int k = 0; k < 6; k++) ob[k] = make_double2(w[k].re, w[k].im);
    a = pa.at(0, j) + r * fstride;
    for (int k = 0; k < 12; k++) v[k] = ld_any(x + a + k * pa.cstride);
    project<3, +1>(v, h);
    double2 *of = own_f + ((int64_t)r * pa.Ls + j) * 6;
    for (int k = 0; k < 6; k++) of[k] = make_double2(h[k].re, h[k].im);
}

// out at plane 0 += coef * (1 + gamma_t)-reconstruction of (received - own) backward hops;
// out at plane lt-1 += coef * (1 - gamma_t)-reconstruction of U_t (received - own) projections
__global__ void __launch_bounds__(128) k_slab_fix(double2 *out, PlaneAddr pa, int64_t fstride, const double2 *U,
                                                  const int64_t *last_link, int64_t lstride, int nrhs, double coef,
                                                  const double2 *own_b, const double2 *own_f, const double2 *got_b,
                                                  const double2 *got_f)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y >> 1, plane = blockIdx.y & 1;
    if (j >= pa.Ls || r >= nrhs) return;
    const int64_t o = ((int64_t)r * pa.Ls + j) * 6;
    cpx<double> h[6], acc[12];
    for (int k = 0; k < 12; k++) acc[k] = mk(0.0, 0.0);
    if (plane == 0) {
        for (int k = 0; k < 6; k++) {
            double2 a = got_b[o + k], b = own_b[o + k];
            h[k] = mk(a.x - b.x, a.y - b.y);
        }
        reconstruct_add<3, -1>(h, acc);
    } else {
        cpx<double> u[9], w[6];
        for (int k = 0; k < 6; k++) {
            double2 a = got_f[o + k], b = own_f[o + k];
            h[k] = mk(a.x - b.x, a.y - b.y);
        }
        const int64_t lb = __ldg(last_link + j);
        for (int k = 0; k < 9; k++) {
            double2 e = __ldg(U + lb + k * lstride);
            u[k] = mk(e.x, e.y);
        }
        su3_mul_half<false>(u, h, w);
        reconstruct_add<3, +1>(w, acc);
    }
    double2 *y = out + pa.at(plane, j) + r * fstride;
    for (int k = 0; k < 12; k++) {
        double2 v = y[k * pa.cstride];
        y[k * pa.cstride] = make_double2(v.x + coef * acc[k].re, v.y + coef * acc[k].im);
    }
}

qdd_status slab_dslash_begin(Gauge *g, const void *in, bool in_f32, bool host_layout, int nrhs, cudaStream_t s)
{
    if (!g->slab) return QDD_OK;
    Slab &sl = *g->slab;
    const HostGeom &hg = g->hg;
    const size_t per = (size_t)nrhs * sl.Ls * 6;  // double2 of one buffer
    if (sl.buf_rhs < (size_t)nrhs) {
        QDD_CUDA(cudaStreamSynchronize(sl.side));
        QDD_TRY(sl.bufs.alloc(g->ctx, 4 * per * sizeof(double2)));
        sl.buf_rhs = nrhs;
    }
    const size_t bytes = per * sizeof(double2);
    QDD_TRY(ensure_host(sl, sl.host_op, sl.op_bytes, 4 * bytes));
    double2 *own_b = sl.bufs.as<double2>(), *own_f = own_b + per;
    sl.op_host_layout = host_layout;
    PlaneAddr pa{host_layout ? nullptr : sl.plane_base.as<int64_t>(), host_layout ? 1 : (int64_t)hg.Vd, sl.Ls, sl.lt};
    const int64_t fstride = (int64_t)hg.V * 12;
    dim3 grid((sl.Ls + 127) / 128, nrhs);
    // the input is complete in stream s's order
    QDD_CUDA(cudaEventRecord(sl.ev_in, s));
    QDD_CUDA(cudaStreamWaitEvent(sl.side, sl.ev_in, 0));
    g->ctx->timer.count(K_OTHER);
    if (in_f32)
        k_slab_pack<float2><<<grid, 128, 0, sl.side>>>((const float2 *)in, pa, fstride, g->links64.as<double2>(),
                                                       sl.last_link.as<int64_t>(), hg.Vd, nrhs, own_b, own_f);
    else
        k_slab_pack<double2><<<grid, 128, 0, sl.side>>>((const double2 *)in, pa, fstride, g->links64.as<double2>(),
                                                        sl.last_link.as<int64_t>(), hg.Vd, nrhs, own_b, own_f);
    QDD_CUDA(cudaGetLastError());
    // own_b, own_f adjacent: one copy
    QDD_CUDA(cudaMemcpyAsync(sl.host_op, own_b, 2 * bytes, cudaMemcpyDeviceToHost, sl.side));
    return QDD_OK;
}

qdd_status slab_dslash_end(Gauge *g, double2 *out, bool residual, int nrhs, cudaStream_t s)
{
    if (!g->slab) return QDD_OK;
    Slab &sl = *g->slab;
    const HostGeom &hg = g->hg;
    const size_t per = (size_t)nrhs * sl.Ls * 6;
    const size_t bytes = per * sizeof(double2);
    double2 *own_b = sl.bufs.as<double2>(), *own_f = own_b + per, *got_b = own_b + 2 * per, *got_f = own_b + 3 * per;
    char *h = (char *)sl.host_op;
    QDD_CUDA(cudaStreamSynchronize(sl.side));  // packed planes on the host; the operator may still run
    QDD_TRY(shift(sl, h, h + 2 * bytes, h + bytes, h + 3 * bytes, bytes));
    QDD_CUDA(cudaMemcpyAsync(got_b, h + 2 * bytes, 2 * bytes, cudaMemcpyHostToDevice, sl.side));
    QDD_CUDA(cudaEventRecord(sl.ev_out, sl.side));
    QDD_CUDA(cudaStreamWaitEvent(s, sl.ev_out, 0));
    PlaneAddr pa{sl.op_host_layout ? nullptr : sl.plane_base.as<int64_t>(), sl.op_host_layout ? 1 : (int64_t)hg.Vd,
                 sl.Ls, sl.lt};
    g->ctx->timer.count(K_OTHER);
    dim3 grid2((sl.Ls + 127) / 128, 2 * nrhs);
    k_slab_fix<<<grid2, 128, 0, s>>>(out, pa, (int64_t)hg.V * 12, g->links64.as<double2>(),
                                     sl.last_link.as<int64_t>(), hg.Vd, nrhs, residual ? g->kappa : -g->kappa, own_b,
                                     own_f, got_b, got_f);
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

// ------------------------------------------------------------------ clover

__global__ void k_slab_clover(const double2 *ea, const double2 *es, const int *map, int V, int Vd, double2 *a,
                              double2 *sa)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    const int j = __ldg(map + i);
    const int64_t src = (int64_t)(j / Vd) * 36 * Vd + j % Vd, dst = (int64_t)(i / Vd) * 36 * Vd + i % Vd;
    for (int p = 0; p < 36; p++) {
        a[dst + (int64_t)p * Vd] = ea[src + (int64_t)p * Vd];
        sa[dst + (int64_t)p * Vd] = es[src + (int64_t)p * Vd];
    }
}

qdd_status slab_clover_remap(Gauge *g, cudaStream_t s)
{
    Slab &sl = *g->slab;
    const HostGeom &hg = g->hg;
    g->ctx->timer.count(K_OTHER);
    k_slab_clover<<<(hg.V + 127) / 128, 128, 0, s>>>(sl.ext->clov64.as<double2>(), sl.ext->sclov64.as<double2>(),
                                                      sl.ext_map.as<int>(), hg.V, hg.Vd, g->clov64.as<double2>(),
                                                      g->sclov64.as<double2>());
    QDD_CUDA(cudaGetLastError());
    return QDD_OK;
}

// ------------------------------------------------------------------- setup

qdd_status slab_setup(Gauge *g, qdd_gauge *ext, const qdd_comm &comm)
{
    const HostGeom &hg = g->hg, &he = ext->hg;
    std::unique_ptr<Slab> sl(new Slab());
    sl->comm = comm;
    sl->ext = ext;
    sl->lt = hg.L[3];
    sl->Ls = hg.L[0] * hg.L[1] * hg.L[2];
    const int Ls = sl->Ls, dt = hg.dom[3];
    std::vector<int> inv((size_t)hg.V), inv_e((size_t)he.V);
    for (int i = 0; i < hg.V; i++) inv[hg.site_of[i]] = i;
    for (int i = 0; i < he.V; i++) inv_e[he.site_of[i]] = i;
    std::vector<int> map((size_t)hg.V);
    for (int i = 0; i < hg.V; i++) map[i] = inv_e[(size_t)hg.site_of[i] + (size_t)dt * Ls];
    std::vector<int64_t> base(2 * (size_t)Ls), link((size_t)Ls);
    for (int p = 0; p < 2; p++)
        for (int j = 0; j < Ls; j++) {
            const int n = j + (p ? (sl->lt - 1) * Ls : 0), i = inv[n];
            const int64_t d = i / hg.Vd, si = i % hg.Vd;
            base[(size_t)p * Ls + j] = d * 12 * hg.Vd + si;
            if (p) link[j] = (d * 36 + 27) * hg.Vd + si;  // U_t: planes 27..35
        }
    Ctx *c = g->ctx;
    QDD_TRY(sl->ext_map.alloc(c, map.size() * sizeof(int)));
    QDD_TRY(sl->plane_base.alloc(c, base.size() * sizeof(int64_t)));
    QDD_TRY(sl->last_link.alloc(c, link.size() * sizeof(int64_t)));
    QDD_CUDA(cudaMemcpy(sl->ext_map.p, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(sl->plane_base.p, base.data(), base.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(sl->last_link.p, link.data(), link.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    QDD_CUDA(cudaStreamCreateWithFlags(&sl->side, cudaStreamNonBlocking));
    QDD_CUDA(cudaEventCreateWithFlags(&sl->ev_in, cudaEventDisableTiming));
    QDD_CUDA(cudaEventCreateWithFlags(&sl->ev_out, cudaEventDisableTiming));
    g->slab = std::move(sl);
    return QDD_OK;
}

}  // namespace qdd

using namespace qdd;

extern "C" qdd_status qdd_slab_regions(const int Lloc[4], const int dom[4], int colour, int out[6])
{
    clear_error();
    if (!Lloc || !dom || !out || (colour != 0 && colour != 1)) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    HostGeom hg;
    QDD_TRY(make_geometry(Lloc, dom, hg));
    slab_regions(hg, colour, out);
    return QDD_OK;
}

extern "C" qdd_status qdd_layout_faces(const int L[4], const int dom[4], int foff[8], uint32_t *fcoord)
{
    clear_error();
    if (!L || !dom) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    HostGeom hg;
    QDD_TRY(make_geometry(L, dom, hg));
    if (foff) std::memcpy(foff, hg.foff, sizeof(hg.foff));
    if (fcoord) std::memcpy(fcoord, hg.fcoord.data(), hg.fcoord.size() * sizeof(uint32_t));
    return QDD_OK;
}
