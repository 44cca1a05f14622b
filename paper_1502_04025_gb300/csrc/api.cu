// C ABI of libqdd: contexts, gauge fields, operator and preconditioner
// entry points, and host-side helpers (arXiv:1502.04025, Sec. 3).
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace qdd {

// ------------------------------------------------------------------ errors

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// ------------------------------------------------------------------ timing

cudaEvent_t Timer::get_event()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Timer::begin(int cls, cudaStream_t s, cudaEvent_t *a)
{
    std::lock_guard<std::mutex> lk(mu);
    launches[cls]++;
    if (mask & (1 << cls)) {
        *a = get_event();
        cudaEventRecord(*a, s);
    }
}

void Timer::begin_seq(int cls, cudaStream_t s, cudaEvent_t *a)
{
    std::lock_guard<std::mutex> lk(mu);
    if (mask & (1 << cls)) {
        *a = get_event();
        cudaEventRecord(*a, s);
    }
}

void Timer::count(int cls)
{
    std::lock_guard<std::mutex> lk(mu);
    launches[cls]++;
}

void Timer::work(int cls, double f, double b)
{
    std::lock_guard<std::mutex> lk(mu);
    flop[cls] += f;
    bytes[cls] += b;
}

void Timer::end(int cls, cudaStream_t s, cudaEvent_t a)
{
    if (!a) return;
    std::lock_guard<std::mutex> lk(mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, s);
    pending.push_back({a, b, cls});
}

void Timer::resolve()
{
    std::lock_guard<std::mutex> lk(mu);
    std::vector<Pending> keep;
    for (auto &p : pending) {
        if (cudaEventQuery(p.b) != cudaSuccess) {
            keep.push_back(p);
            continue;
        }
        float t = 0;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
            ms[p.cls] += t;
            timed[p.cls]++;
        }
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.swap(keep);
    cudaGetLastError();
}

Timer::~Timer()
{
    for (auto &p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

// ------------------------------------------------------------------ memory

qdd_status DevMem::alloc(Ctx *c, size_t n)
{
    release();
    if (n == 0) return QDD_OK;
    if (c->used.load() + n > c->budget) {
        set_error("allocation of %zu bytes exceeds the HBM budget (%zu of %zu bytes in use)", n, c->used.load(),
                  c->budget);
        return QDD_EBUDGET;
    }
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        return QDD_ENOMEM;
    }
    ctx = c;
    bytes = n;
    c->used += n;
    return QDD_OK;
}

void DevMem::release()
{
    if (p) {
        cudaFree(p);
        if (ctx) ctx->used -= bytes;
    }
    p = nullptr;
    bytes = 0;
}

// -------------------------------------------------------- precision copies

static size_t elem_bytes(qdd_prec p)
{
    switch (p) {
    case QDD_PREC_F64: return 16;
    case QDD_PREC_DF64: return 16;
    case QDD_PREC_F32: return 8;
    default: return 4;
    }
}

qdd_status ensure_copy(Gauge *g, qdd_prec prec, cudaStream_t s)
{
    if (prec == QDD_PREC_F64) return QDD_OK;
    if (prec == QDD_PREC_H16) return ensure_copy(g, QDD_PREC_F16S, s);
    if (prec < QDD_PREC_F64 || prec > QDD_PREC_DF64) {
        set_error("invalid precision %d", (int)prec);
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->copy_mu);
    PrecCopy &c = g->copies[prec];
    if (c.valid) return QDD_OK;
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    if (prec == QDD_PREC_DF64) {
        // links and clover split into hi + lo FP32 parts (the operator only)
        const size_t n = (size_t)g->hg.V * 36;
        QDD_TRY(c.links.ensure(g->ctx, n * sizeof(float4)));
        QDD_TRY(c.clov.ensure(g->ctx, n * sizeof(float4)));
        QDD_TRY(launch_split_convert(g, g->links64.as<double2>(), c.links.as<float4>(), (int64_t)n, s));
        QDD_TRY(launch_split_convert(g, g->clov64.as<double2>(), c.clov.as<float4>(), (int64_t)n, s));
        c.valid = true;
        return QDD_OK;
    }
    const size_t V = g->hg.V, eb = elem_bytes(prec);
    const bool scaled = prec == QDD_PREC_F16S || prec == QDD_PREC_BF16S;
    QDD_TRY(c.links.ensure(g->ctx, V * 36 * eb));
    QDD_TRY(c.clov.ensure(g->ctx, V * 36 * eb));
    QDD_TRY(c.sclov.ensure(g->ctx, V * 36 * eb));
    if (scaled) {
        QDD_TRY(c.clov_s.ensure(g->ctx, V * 4));
        QDD_TRY(c.sclov_s.ensure(g->ctx, V * 4));
    }
    QDD_TRY(launch_links_convert(g, prec, c.links.p, s));
    QDD_TRY(launch_clover_convert(g, g->clov64.as<double2>(), prec, c.clov.p, c.clov_s.as<float>(), s, true));
    QDD_TRY(launch_clover_convert(g, g->sclov64.as<double2>(), prec, c.sclov.p, c.sclov_s.as<float>(), s));
    c.valid = true;
    return QDD_OK;
}

qdd_status ensure_links12(Gauge *g, qdd_prec prec, cudaStream_t s)
{
    prec = field_store(prec);
    if (prec != QDD_PREC_F32 && prec != QDD_PREC_F16S && prec != QDD_PREC_BF16S) {
        set_error("two-row links exist for FP32, FP16 and BF16 storage only");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->copy_mu);
    PrecCopy &c = g->copies[prec];
    if (c.valid12) return QDD_OK;
    QDD_TRY(c.links12.ensure(g->ctx, (size_t)g->hg.V * 24 * elem_bytes(prec)));
    QDD_TRY(launch_links12_convert(g, prec, c.links12.p, s));
    c.valid12 = true;
    return QDD_OK;
}

// per-gauge staging buffers for the entry points that are not the solver
struct Staging {
    DevMem io, a, a_s, b, b_s, c, c_s, err;
};

Gauge::~Gauge() = default;

static qdd_status stage_in(Gauge *g, DevMem &io, const double *src, int nrhs, int on_device, cudaStream_t s,
                           const double **dev)
{
    size_t bytes = (size_t)g->hg.V * 24 * sizeof(double) * nrhs;
    if (on_device) {
        *dev = src;
        return QDD_OK;
    }
    QDD_TRY(io.ensure(g->ctx, bytes));
    QDD_CUDA(cudaMemcpyAsync(io.p, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = io.as<double>();
    return QDD_OK;
}

static qdd_status stage_out(Gauge *g, DevMem &io, double *dst, int nrhs, int on_device, cudaStream_t s,
                            double **dev)
{
    size_t bytes = (size_t)g->hg.V * 24 * sizeof(double) * nrhs;
    if (on_device) {
        *dev = dst;
        return QDD_OK;
    }
    QDD_TRY(io.ensure(g->ctx, bytes));
    *dev = io.as<double>();
    return QDD_OK;
}

static qdd_status finish_out(Gauge *g, DevMem &io, double *dst, int nrhs, int on_device, cudaStream_t s)
{
    size_t bytes = (size_t)g->hg.V * 24 * sizeof(double) * nrhs;
    if (!on_device) QDD_CUDA(cudaMemcpyAsync(dst, io.p, bytes, cudaMemcpyDeviceToHost, s));
    QDD_CUDA(cudaStreamSynchronize(s));
    g->ctx->timer.resolve();
    return QDD_OK;
}

}  // namespace qdd

using namespace qdd;

// ======================================================================= C ABI

extern "C" {

const char *qdd_last_error(void) { return g_err; }

qdd_status qdd_create(qdd_ctx **out, int device, size_t hbm_budget_bytes)
{
    clear_error();
    if (!out) {
        set_error("ctx is NULL");
        return QDD_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    QDD_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("device %d out of range (%d devices)", device, ndev);
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaSetDevice(device));
    size_t free_b = 0, total_b = 0;
    QDD_CUDA(cudaMemGetInfo(&free_b, &total_b));
    qdd_ctx *c = new qdd_ctx();
    c->device = device;
    QDD_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device));
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)total_b);
    *out = c;
    return QDD_OK;
}

qdd_status qdd_set_profiling(qdd_ctx *ctx, int classes)
{
    if (!ctx) return QDD_EINVAL;
    QDD_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    ctx->timer.mask = classes & QDD_PROF_ALL;
    // create the events up front so that timed regions create none
    while (classes && ctx->timer.pool.size() < 4096) {
        cudaEvent_t e = nullptr;
        QDD_CUDA(cudaEventCreate(&e));
        ctx->timer.pool.push_back(e);
    }
    return QDD_OK;
}

qdd_status qdd_get_kernel_times(qdd_ctx *ctx, double out[6], int reset)
{
    if (!ctx || !out) return QDD_EINVAL;
    cudaSetDevice(ctx->device);
    ctx->timer.resolve();
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    for (int c = 0; c < 3; c++) {
        out[2 * c] = ctx->timer.ms[c];
        out[2 * c + 1] = (double)ctx->timer.launches[c];
    }
    if (reset)
        for (int c = 0; c < 4; c++) {
            ctx->timer.ms[c] = 0;
            ctx->timer.launches[c] = 0;
            ctx->timer.timed[c] = 0;
            ctx->timer.flop[c] = 0;
            ctx->timer.bytes[c] = 0;
        }
    return QDD_OK;
}

qdd_status qdd_get_kernel_work(qdd_ctx *ctx, double out[6])
{
    if (!ctx || !out) return QDD_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    for (int c = 0; c < 3; c++) {
        out[2 * c] = ctx->timer.flop[c];
        out[2 * c + 1] = ctx->timer.bytes[c];
    }
    return QDD_OK;
}

qdd_status qdd_memory(qdd_ctx *ctx, size_t *used, size_t *budget)
{
    if (!ctx) return QDD_EINVAL;
    if (used) *used = ctx->used.load();
    if (budget) *budget = ctx->budget;
    return QDD_OK;
}

qdd_status qdd_create_gauge_field(qdd_ctx *ctx, const int L[4], const int dom[4], const double *links,
                                  int links_on_device, qdd_gauge **out)
{
    clear_error();
    if (!ctx || !L || !dom || !links || !out) {
        set_error("null argument");
        return QDD_EINVAL;
    }
    *out = nullptr;
    QDD_CUDA(cudaSetDevice(ctx->device));
    std::unique_ptr<qdd_gauge> g(new qdd_gauge());
    g->ctx = ctx;
    QDD_TRY(make_geometry(L, dom, g->hg));
    const HostGeom &hg = g->hg;
    QDD_TRY(g->d_nbl.alloc(ctx, hg.nbl.size() * sizeof(uint16_t)));
    QDD_TRY(g->d_nbd.alloc(ctx, hg.nbd.size() * sizeof(int)));
    QDD_TRY(g->d_site_of.alloc(ctx, hg.site_of.size() * sizeof(int)));
    QDD_TRY(g->d_block_slot.alloc(ctx, hg.block_slot.size() * sizeof(int)));
    QDD_TRY(g->d_fcoord.alloc(ctx, hg.fcoord.size() * sizeof(uint32_t)));
    QDD_CUDA(cudaMemcpy(g->d_fcoord.p, hg.fcoord.data(), hg.fcoord.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(g->d_block_slot.p, hg.block_slot.data(), hg.block_slot.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(g->d_nbl.p, hg.nbl.data(), hg.nbl.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(g->d_nbd.p, hg.nbd.data(), hg.nbd.size() * sizeof(int), cudaMemcpyHostToDevice));
    QDD_CUDA(cudaMemcpy(g->d_site_of.p, hg.site_of.data(), hg.site_of.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    Geom &G = g->geom;
    for (int mu = 0; mu < 4; mu++) {
        G.L[mu] = hg.L[mu];
        G.dom[mu] = hg.dom[mu];
        G.nb[mu] = hg.nb[mu];
    }
    G.V = hg.V;
    G.Vd = hg.Vd;
    G.Vh = hg.Vh;
    G.Nd = hg.Nd;
    G.Nd2 = hg.Nd2;
    G.vd_shift = -1;
    for (int k = 0; k < 31; k++)
        if ((1 << k) == hg.Vd) G.vd_shift = k;
    G.nbl = g->d_nbl.as<uint16_t>();
    G.nbd = g->d_nbd.as<int>();
    G.block_slot = g->d_block_slot.as<int>();
    G.fcoord = g->d_fcoord.as<uint32_t>();
    for (int k = 0; k < 8; k++) G.foff[k] = hg.foff[k];
    G.nf = hg.nf;

    const size_t lbytes = (size_t)hg.V * 36 * sizeof(double2);
    QDD_TRY(g->links64.alloc(ctx, lbytes));
    const double *src = links;
    DevMem tmp;
    if (!links_on_device) {
        QDD_TRY(tmp.alloc(ctx, lbytes));
        QDD_CUDA(cudaMemcpy(tmp.p, links, lbytes, cudaMemcpyHostToDevice));
        src = tmp.as<double>();
    }
    QDD_TRY(launch_links_to_internal(g.get(), src, 0));
    // SU(3) links (to rounding) let the full-lattice operator read two rows per link
    DevMem bad;
    QDD_TRY(bad.alloc(ctx, sizeof(int)));
    QDD_TRY(launch_su3_check(g.get(), kSu3Tol, bad.as<int>(), 0));
    int h_bad = 1;
    QDD_CUDA(cudaMemcpy(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost));
    g->su3 = h_bad == 0;
    g->two_rows = g->su3;
    QDD_CUDA(cudaDeviceSynchronize());
    ctx->timer.resolve();
    *out = g.release();
    return QDD_OK;
}

qdd_status qdd_create_gauge_field_slab(qdd_ctx *ctx, const int Lloc[4], const int dom[4], const double *links_ext,
                                       int links_on_device, const qdd_comm *comm, qdd_gauge **out)
{
    clear_error();
    if (!ctx || !Lloc || !dom || !links_ext || !comm || !out) {
        set_error("null argument");
        return QDD_EINVAL;
    }
    *out = nullptr;
    if (comm->size < 1 || comm->rank < 0 || comm->rank >= comm->size || !comm->allreduce_sum || !comm->shift) {
        set_error("invalid communication hooks (rank %d of %d)", comm->rank, comm->size);
        return QDD_EINVAL;
    }
    if (dom[3] < 2) {
        set_error("invalid domain extent in t");
        return QDD_EINVAL;
    }
    const int Le[4] = {Lloc[0], Lloc[1], Lloc[2], Lloc[3] + 2 * dom[3]};
    const size_t Ls = (size_t)Lloc[0] * Lloc[1] * Lloc[2];
    // the owned planes start dom[3] planes into the extended field (t is the slowest index)
    const double *own = links_ext + (size_t)dom[3] * Ls * 4 * 18;
    qdd_gauge *g = nullptr, *e = nullptr;
    QDD_TRY(qdd_create_gauge_field(ctx, Lloc, dom, own, links_on_device, &g));
    qdd_status st = qdd_create_gauge_field(ctx, Le, dom, links_ext, links_on_device, &e);
    if (st == QDD_OK) st = slab_setup(g, e, *comm);
    if (st != QDD_OK) {
        if (!g->slab) qdd_destroy_gauge(e);
        qdd_destroy_gauge(g);
        return st;
    }
    *out = g;
    return QDD_OK;
}

void qdd_destroy_gauge(qdd_gauge *g)
{
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaDeviceSynchronize();
    delete g;
}

qdd_status qdd_set_link_compression(qdd_gauge *g, int two_rows)
{
    clear_error();
    if (!g || (two_rows != 0 && two_rows != 1)) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    if (two_rows && !g->su3) {
        set_error("links are not SU(3) to %g: the third row cannot be rebuilt from the first two", kSu3Tol);
        return QDD_EINVAL;
    }
    g->two_rows = two_rows != 0;
    return QDD_OK;
}

qdd_status qdd_check_hits(unsigned long long *hits)
{
    clear_error();
    if (!hits) {
        set_error("null argument");
        return QDD_EINVAL;
    }
#ifdef QDD_CHECK
    *hits = check_hits_sap() + check_hits_dslash() + check_hits_mg();
    return QDD_OK;
#else
    *hits = 0;
    set_error("this library was built without range checks (QDD_CHECK)");
    return QDD_EINVAL;
#endif
}

qdd_status qdd_set_schwarz_variant(qdd_gauge *g, int variant)
{
    clear_error();
    if (!g || variant < 0 || variant > 3) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    g->sap_variant = variant;
    return QDD_OK;
}

qdd_status qdd_check_set_wait_limit(int device, unsigned spins)
{
    clear_error();
#ifdef QDD_CHECK
    QDD_CUDA(cudaSetDevice(device));
    return set_first_wait_spins_sap(spins);
#else
    (void)device;
    (void)spins;
    set_error("this library was built without range checks (QDD_CHECK)");
    return QDD_EINVAL;
#endif
}

qdd_status qdd_link_compression(qdd_gauge *g, int *two_rows, int *is_su3)
{
    clear_error();
    if (!g || !two_rows || !is_su3) {
        set_error("null argument");
        return QDD_EINVAL;
    }
    *two_rows = g->two_rows ? 1 : 0;
    *is_su3 = g->su3 ? 1 : 0;
    return QDD_OK;
}

qdd_status qdd_set_clover(qdd_gauge *g, double c_sw, double kappa)
{
    clear_error();
    if (!g) return QDD_EINVAL;
    if (!std::isfinite(c_sw) || !std::isfinite(kappa)) {
        set_error("c_sw and kappa must be finite");
        return QDD_EINVAL;
    }
    // a sharded field takes the clover of its owned sites from its extended
    // lattice, whose halo holds the links the boundary planes' leaves need
    qdd_status ext_st = g->slab ? qdd_set_clover(g->slab->ext, c_sw, kappa) : QDD_OK;
    std::lock_guard<std::mutex> lk(g->mu);
    QDD_CUDA(cudaSetDevice(g->ctx->device));
    const size_t cb = (size_t)g->hg.V * 36 * sizeof(double2);
    QDD_TRY(g->clov64.ensure(g->ctx, cb));
    QDD_TRY(g->sclov64.ensure(g->ctx, cb));
    int singular = 0;
    if (g->slab) {
        g->have_clover = false;
        if (ext_st != QDD_OK) return ext_st;
        QDD_TRY(slab_clover_remap(g, 0));
        QDD_CUDA(cudaDeviceSynchronize());
    } else {
        DevMem flag;
        QDD_TRY(flag.alloc(g->ctx, sizeof(int)));
        QDD_CUDA(cudaMemset(flag.p, 0, sizeof(int)));
        QDD_TRY(launch_clover_build(g, c_sw, kappa, flag.as<int>(), 0));
        QDD_CUDA(cudaMemcpy(&singular, flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    }
    g->ctx->timer.resolve();
    for (int p = 0; p < 5; p++) g->copies[p].valid = false;
    g->have_clover = false;
    if (singular) {
        set_error("clover block singular on %d sites", singular);
        return QDD_EINVAL;
    }
    g->csw = c_sw;
    g->kappa = kappa;
    g->have_clover = true;
    return QDD_OK;
}

qdd_status qdd_get_clover(qdd_gauge *g, int which, double *out)
{
    clear_error();
    if (!g || !out || (which != 0 && which != 1)) return QDD_EINVAL;
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaSetDevice(g->ctx->device));
    const HostGeom &hg = g->hg;
    std::vector<double2> buf((size_t)hg.V * 36);
    QDD_CUDA(cudaMemcpy(buf.data(), (which ? g->sclov64 : g->clov64).p, buf.size() * sizeof(double2),
                        cudaMemcpyDeviceToHost));
    for (int gi = 0; gi < hg.V; gi++) {
        int d = gi / hg.Vd, s = gi % hg.Vd;
        int n = hg.site_of[gi];
        for (int blk = 0; blk < 2; blk++) {
            const double2 *p = buf.data() + ((size_t)d * 36 + blk * 18) * hg.Vd + s;
            double *o = out + ((size_t)n * 2 + blk) * 72;  // 36 complex
            double diag[6] = {p[0].x, p[0].y, p[(size_t)hg.Vd].x, p[(size_t)hg.Vd].y, p[(size_t)2 * hg.Vd].x,
                              p[(size_t)2 * hg.Vd].y};
            for (int i = 0; i < 6; i++) {
                o[(i * 6 + i) * 2] = diag[i];
                o[(i * 6 + i) * 2 + 1] = 0;
            }
            int k = 3;
            for (int i = 0; i < 6; i++)
                for (int j = i + 1; j < 6; j++) {
                    double2 v = p[(size_t)k * hg.Vd];
                    o[(i * 6 + j) * 2] = v.x;
                    o[(i * 6 + j) * 2 + 1] = v.y;
                    o[(j * 6 + i) * 2] = v.x;
                    o[(j * 6 + i) * 2 + 1] = -v.y;
                    k++;
                }
        }
    }
    return QDD_OK;
}

qdd_status qdd_apply_D(qdd_gauge *g, const double *in, double *out, int nrhs, qdd_prec prec, int on_device,
                       void *stream)
{
    clear_error();
    if (!g || !in || !out || nrhs < 1 || prec < QDD_PREC_F64 || prec > QDD_PREC_H16) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    QDD_CUDA(cudaSetDevice(g->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    auto &st = g->stage;  // under g->mu
    if (!st) st.reset(new Staging());
    const size_t V = g->hg.V;
    const size_t eb = elem_bytes(spinor_store(prec));
    const bool scaled = prec == QDD_PREC_F16S || prec == QDD_PREC_BF16S;
    const qdd_prec arith = prec == QDD_PREC_F64 || prec == QDD_PREC_DF64 ? prec : QDD_PREC_F32;
    const qdd_prec fp = field_store(prec);                                // link / clover copy
    if (prec == QDD_PREC_DF64) prec = QDD_PREC_F64;                       // spinor storage
    prec = spinor_store(prec);
    const double *din = nullptr;
    double *dout = nullptr;
    QDD_TRY(stage_in(g, st->io, in, nrhs, on_device, s, &din));
    QDD_TRY(st->a.ensure(g->ctx, V * 12 * eb * nrhs));
    QDD_TRY(st->b.ensure(g->ctx, V * 12 * eb * nrhs));
    if (scaled) {
        QDD_TRY(st->a_s.ensure(g->ctx, V * 4 * nrhs));
        QDD_TRY(st->b_s.ensure(g->ctx, V * 4 * nrhs));
    }
    QDD_TRY(launch_spinor_in(g, din, st->a.p, st->a_s.as<float>(), prec, nrhs, s));
    // a sharded field: its boundary planes (FP64, host layout) move while the operator runs
    QDD_TRY(slab_dslash_begin(g, din, false, true, nrhs, s));
    QDD_TRY(launch_dslash(g, arith, fp, st->a.p, st->a_s.as<float>(), prec, st->b.p, st->b_s.as<float>(), prec,
                          nullptr, nrhs, s));
    // a sharded field corrects the output's boundary planes from the input
    // (FP64, host layout), so the host output must not reuse the input's staging
    DevMem &oio = g->slab ? st->c : st->io;
    if (g->slab && on_device && out == in) {
        set_error("a sharded field needs separate input and output buffers");
        return QDD_EINVAL;
    }
    QDD_TRY(stage_out(g, oio, out, nrhs, on_device, s, &dout));
    QDD_TRY(launch_spinor_out(g, st->b.p, st->b_s.as<float>(), dout, prec, nrhs, s));
    QDD_TRY(slab_dslash_end(g, (double2 *)dout, false, nrhs, s));
    return finish_out(g, oio, out, nrhs, on_device, s);
}

qdd_status qdd_sap_apply(qdd_gauge *g, const double *eta, double *psi, double *rho, int nrhs, int nmr, int n_half,
                         qdd_prec prec, int on_device, void *stream)
{
    clear_error();
    if (!g || !eta || !psi || nrhs < 1 || nmr < 0 || n_half < 1 || !is_sap_prec(prec)) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    QDD_CUDA(cudaSetDevice(g->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    auto &st = g->stage;  // under g->mu
    if (!st) st.reset(new Staging());
    const size_t V = g->hg.V;
    const qdd_prec ssp = spinor_store(prec);                                 // rho storage
    const size_t eb = elem_bytes(ssp);
    const qdd_prec pp = prec == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;  // psi storage
    const bool scaled = prec == QDD_PREC_F16S || prec == QDD_PREC_BF16S;
    const double *din = nullptr;
    QDD_TRY(stage_in(g, st->io, eta, nrhs, on_device, s, &din));
    QDD_TRY(st->a.ensure(g->ctx, V * 12 * eb * nrhs));                  // rho
    QDD_TRY(st->b.ensure(g->ctx, sap_face_bytes(g->hg, prec, nrhs)));   // face slots
    QDD_TRY(st->c.ensure(g->ctx, V * 12 * elem_bytes(pp) * nrhs));      // psi
    QDD_TRY(st->err.ensure(g->ctx, sizeof(int)));
    if (scaled) QDD_TRY(st->a_s.ensure(g->ctx, V * 4 * nrhs));
    QDD_CUDA(cudaMemsetAsync(st->err.p, 0, sizeof(int), s));
    QDD_TRY(launch_spinor_in(g, din, st->a.p, st->a_s.as<float>(), ssp, nrhs, s));
    if (n_half < 2) QDD_CUDA(cudaMemsetAsync(st->c.p, 0, V * 12 * elem_bytes(pp) * nrhs, s));
    SapBuffers b{st->a.p, st->b.p, st->c.p, st->a_s.as<float>()};
    {
        SeqScope seq(g->ctx->timer, K_SAP, s);
        for (int hs = 0; hs < n_half; hs++) {
            // a sharded field exchanges the face slots that cross its slab
            // boundaries while the interior domains are swept
            if (g->slab)
                QDD_TRY(slab_sap_halfsweep(g, prec, b, hs & 1, nmr, nrhs, hs < 2, hs >= 1, st->err.as<int>(), s,
                                           hs + 1 < n_half || rho));
            else
                QDD_TRY(launch_sap_halfsweep(g, prec, b, hs & 1, nmr, nrhs, hs < 2, hs >= 1, 0, st->err.as<int>(), s,
                                             hs >= 1, false));
        }
    }
    if (rho)  // bring the residual of the next colour up to date
        QDD_TRY(launch_sap_halfsweep(g, prec, b, n_half & 1, nmr, nrhs, 0, 1, 1, st->err.as<int>(), s));
    double *dout = nullptr;
    QDD_TRY(stage_out(g, st->io, psi, nrhs, on_device, s, &dout));
    QDD_TRY(launch_spinor_out(g, st->c.p, nullptr, dout, pp, nrhs, s));
    QDD_TRY(finish_out(g, st->io, psi, nrhs, on_device, s));
    if (rho) {
        QDD_TRY(stage_out(g, st->io, rho, nrhs, on_device, s, &dout));
        QDD_TRY(launch_spinor_out(g, st->a.p, st->a_s.as<float>(), dout, ssp, nrhs, s));
        QDD_TRY(finish_out(g, st->io, rho, nrhs, on_device, s));
    }
    int err = 0;
    QDD_CUDA(cudaMemcpy(&err, st->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("device wait ran out in the Schwarz kernel (flags %d)", err);
        return QDD_ETIMEOUT;
    }
    return QDD_OK;
}

void qdd_default_params(qdd_solve_params *p)
{
    if (!p) return;
    p->tol = 1e-10;
    p->restart_m = 16;
    p->max_restarts = 50;
    p->nmr = 4;
    p->ncy = 4;
    p->sap_prec = QDD_PREC_F32;
    p->arnoldi_prec = QDD_PREC_F64;
    p->use_sap = 1;
    p->nrhs = 1;
    p->reorth = 1;
    p->relax_eta = 0.0;
    p->dr_k = 0;
}

qdd_status qdd_solve(qdd_gauge *g, const double *b, double *x, int on_device, const qdd_solve_params *p,
                     qdd_report *rep, void *stream)
{
    clear_error();
    if (!g || !b || !x || !p) {
        set_error("null argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    QDD_CUDA(cudaSetDevice(g->ctx->device));
    if (!g->ws) g->ws = make_workspace();
    return solve_impl(g, g->ws.get(), b, x, on_device, p, rep, (cudaStream_t)stream);
}

qdd_status qdd_cdot_multi(qdd_ctx *ctx, const double *v, int nvec, int64_t ld, const double *w, int64_t n,
                          double *out, void *stream)
{
    clear_error();
    if (!ctx || !v || !w || !out || nvec < 1 || nvec > 64 || n < 1 || ld < n) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(ctx->red_mu);
    QDD_TRY(blas_scratch_ensure(ctx, ctx->red_scratch));
    QDD_TRY(blas_cdot_multi(ctx, (const double2 *)v, nvec, ld, (const double2 *)w, n, (double2 *)out,
                            ctx->red_scratch.as<double2>(), s));
    QDD_CUDA(cudaStreamSynchronize(s));
    ctx->timer.resolve();
    return QDD_OK;
}

qdd_status qdd_layout(const int L[4], const int dom[4], int *site_of, uint16_t *nbl, int *nbd)
{
    clear_error();
    if (!L || !dom) return QDD_EINVAL;
    HostGeom hg;
    QDD_TRY(make_geometry(L, dom, hg));
    if (site_of) std::memcpy(site_of, hg.site_of.data(), hg.site_of.size() * sizeof(int));
    if (nbl) std::memcpy(nbl, hg.nbl.data(), hg.nbl.size() * sizeof(uint16_t));
    if (nbd) std::memcpy(nbd, hg.nbd.data(), hg.nbd.size() * sizeof(int));
    return QDD_OK;
}

double qdd_load_model(double n_domains_per_colour, double n_slots)
{
    if (!(n_domains_per_colour > 0) || !(n_slots > 0)) return 0.0;
    double x = n_domains_per_colour / n_slots;
    return x / std::ceil(x);
}

double qdd_domain_working_set(const int dom[4], int link_bytes, int n_full, int n_even)
{
    if (!dom) return 0.0;
    double vd = (double)dom[0] * dom[1] * dom[2] * dom[3];
    return vd * ((72.0 + 72.0) * link_bytes + (24.0 * n_full + 12.0 * n_even) * 4.0);
}

}  // extern "C"
