// Serving loop: asynchronous solves with admission by the HBM budget and
// continuous batching.
//
// Requests queue on the context.  Worker threads (one CUDA stream and one
// Krylov workspace each; max_slots of them) take the oldest request together
// with every queued request for the same gauge field and parameters (up to
// 12 right-hand sides) once everything their solve allocates fits in the
// budget next to what is already resident (allocated at admission, under
// the queue lock), and solve them as one multi-right-hand-side batch:
// one Schwarz launch per half-sweep covers all of them and reuses each staged
// domain for every source.  Requests of different workers run concurrently
// on the device.  Each right-hand side's arithmetic (Schwarz block solves,
// operator, Gram-Schmidt, Givens) is independent of the others in the batch
// and runs with the same launch shapes, so a result does not depend on the
// mix it was solved in.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>

#include "admission.h"
#include "internal.h"

namespace qdd {

constexpr int kMaxBatchRhs = 12;

struct Request {
    uint64_t ticket = 0;
    Gauge *g = nullptr;
    std::unique_ptr<double[]> b;  // the sources, copied at submission
    size_t bn = 0;                // their doubles
    double *x = nullptr;
    qdd_solve_params p{};
    qdd_status status = QDD_OK;
    qdd_report rep{};
    std::vector<double> hist;
    std::string err;
    bool done = false;
    int bypassed = 0;  // later requests admitted while this one waited at the head of the queue
    std::chrono::steady_clock::time_point t_submit;
};

// a request at the head of the queue that does not fit lets at most this many
// later requests that do fit go first; then admission is strictly in order
// until it runs
constexpr int kMaxBypass = 8;

// Host copy of n doubles on several threads: one request's sources reach
// gigabytes (12 spinors of a 32^3x64 lattice: 4.8 GB), which one thread
// copies at a fraction of the host's memory bandwidth, delaying the caller's
// next submission or this worker's next batch.
static void par_copy(double *dst, const double *src, size_t n)
{
    const size_t kChunk = (size_t)1 << 23;  // 64 MB: below this one thread copies
    unsigned hw = std::thread::hardware_concurrency();
    const size_t nt = std::min<size_t>(std::min<size_t>(hw ? hw : 1, 16), (n + kChunk - 1) / kChunk);
    if (nt <= 1) {
        std::memcpy(dst, src, n * sizeof(double));
        return;
    }
    std::vector<std::thread> th;
    const size_t per = (n + nt - 1) / nt;
    for (size_t t = 0; t < nt; t++) {
        const size_t a = t * per, e = std::min(n, a + per);
        if (a < e) th.emplace_back([=] { std::memcpy(dst + a, src + a, (e - a) * sizeof(double)); });
    }
    for (auto &t : th) t.join();
}

static bool same_params(const qdd_solve_params &a, const qdd_solve_params &b)
{
    return a.tol == b.tol && a.restart_m == b.restart_m && a.max_restarts == b.max_restarts && a.nmr == b.nmr &&
           a.ncy == b.ncy && a.sap_prec == b.sap_prec && a.arnoldi_prec == b.arnoldi_prec &&
           a.use_sap == b.use_sap && a.reorth == b.reorth && a.relax_eta == b.relax_eta && a.dr_k == b.dr_k;
}

static void worker_main(Ctx *ctx)
{
    cudaSetDevice(ctx->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::unique_ptr<Workspace> ws = make_workspace();
    std::vector<double> bm, xm;
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lk(ctx->q_mu);
            for (;;) {
                if (ctx->stopping) {
                    lk.unlock();
                    workspace_release(ws.get());
                    cudaStreamDestroy(st);
                    return;
                }
                if (!ctx->queue.empty()) {
                    // admission (the rules: admission.h).  Everything a batch's solve
                    // allocates (workspace, precision copies of the gauge field) is
                    // allocated here, under the lock, so that admissions never count
                    // the same free memory twice.
                    auto prepare = [&](const Request &lead, int total) -> qdd_status {
                        qdd_solve_params pm = lead.p;
                        pm.nrhs = total;
                        const size_t need = workspace_bytes(lead.g, pm.restart_m, total, pm.sap_prec,
                                                            pm.use_sap != 0, pm.dr_k);
                        // a workspace that cannot fit next to everything else is not tried
                        const size_t held = workspace_held(ws.get()), used = ctx->used.load();
                        if ((used > held ? used - held : 0) + need > ctx->budget) return QDD_EBUDGET;
                        if (held > 2 * need) workspace_release(ws.get());
                        clear_error();
                        qdd_status ps = solve_prepare(lead.g, ws.get(), &pm, st);
                        if (ps == QDD_EBUDGET) workspace_release(ws.get());
                        return ps;
                    };
                    auto res = admit(
                        ctx->queue, ctx->running > 0, kMaxBatchRhs, kMaxBypass,
                        [](const Request &r) { return r.p.nrhs; },
                        [](const Request &a, const Request &b) { return a.g == b.g && same_params(a.p, b.p); },
                        prepare);
                    if (res.what == Admit::kBatch) {
                        batch = std::move(res.batch);
                        break;
                    }
                    if (res.what == Admit::kReject) {
                        auto &bad = res.rejected;
                        bad->status = res.status;
                        bad->err = res.status == QDD_EBUDGET ? "request does not fit in the HBM budget"
                                                             : std::string(qdd_last_error());
                        bad->done = true;
                        ctx->done_cv.notify_all();
                        continue;
                    }
                }
                ctx->q_cv.wait(lk);
            }
            ctx->running++;
        }
        // ---- run the batch (a single request solves straight from/to its own buffers)
        const Gauge *g = batch[0]->g;
        const size_t per = (size_t)g->hg.V * 24;
        int total = 0;
        for (auto &r : batch) total += r->p.nrhs;
        const bool single = batch.size() == 1;
        size_t off = 0;
        if (!single) {
            bm.resize(per * total);
            xm.resize(per * total);
            for (auto &r : batch) {
                par_copy(bm.data() + off, r->b.get(), r->bn);
                off += r->bn;
            }
        }
        qdd_solve_params pm = batch[0]->p;
        pm.nrhs = total;
        qdd_report rep{};
        std::vector<double> rel;
        clear_error();
        qdd_status s = single ? solve_impl(batch[0]->g, ws.get(), batch[0]->b.get(), batch[0]->x, 0, &pm, &rep, st,
                                           &rel)
                              : solve_impl(batch[0]->g, ws.get(), bm.data(), xm.data(), 0, &pm, &rep, st, &rel);
        std::string msg = s == QDD_OK ? std::string() : std::string(qdd_last_error());
        auto t_done = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(ctx->q_mu);
            off = 0;
            int r0 = 0;
            for (auto &r : batch) {
                if (!single) par_copy(r->x, xm.data() + off, r->bn);
                off += r->bn;
                r->rep = rep;
                double tr = 0;
                for (int k = 0; k < r->p.nrhs; k++)
                    if (r0 + k < (int)rel.size()) tr = std::max(tr, rel[r0 + k]);
                r->rep.true_rel_res = tr;
                r->rep.converged = (s == QDD_OK || tr <= r->p.tol) ? (tr <= r->p.tol) : 0;
                r->rep.seconds = std::chrono::duration<double>(t_done - r->t_submit).count();
                r->hist.assign(rep.res_history, rep.res_history + rep.n_history);
                r->rep.res_history = nullptr;
                r->status = (s == QDD_ENOCONV && r->rep.converged) ? QDD_OK : s;
                r->err = msg;
                r->done = true;
                r->b.reset();  // the source copy is no longer needed
                r0 += r->p.nrhs;
            }
        }
        ctx->done_cv.notify_all();  // results are out; this worker still counts as running
        // a large idle workspace would block the admission of other requests:
        // give it back (small ones are kept for reuse) before this worker stops
        // counting as running, so that admission never sees an idle device
        // whose memory is still held and rejects a request that would fit
        if (workspace_held(ws.get()) > ((size_t)4 << 30)) workspace_release(ws.get());
        // keep the merge buffers only while they are small
        if (bm.size() > ((size_t)1 << 27)) std::vector<double>().swap(bm);
        if (xm.size() > ((size_t)1 << 27)) std::vector<double>().swap(xm);
        {
            std::lock_guard<std::mutex> lk(ctx->q_mu);
            ctx->running--;
        }
        ctx->q_cv.notify_all();
    }
}

Ctx::~Ctx()
{
    {
        std::lock_guard<std::mutex> lk(q_mu);
        stopping = true;
    }
    q_cv.notify_all();
    for (auto &t : workers) t.join();
}

}  // namespace qdd

using namespace qdd;

extern "C" {

qdd_status qdd_serve_config(qdd_ctx *ctx, int max_slots)
{
    clear_error();
    if (!ctx || max_slots < 1 || max_slots > 64) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if (!ctx->workers.empty()) {
        set_error("the serving loop is already running");
        return QDD_EINVAL;
    }
    ctx->max_slots = max_slots;
    return QDD_OK;
}

qdd_status qdd_submit(qdd_ctx *ctx, qdd_gauge *g, const double *b, double *x, const qdd_solve_params *p,
                      uint64_t *ticket)
{
    clear_error();
    if (!ctx || !g || !b || !x || !p || !ticket || g->ctx != ctx) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    if (p->nrhs < 1 || p->nrhs > kMaxBatchRhs) {
        set_error("nrhs must be 1..%d", kMaxBatchRhs);
        return QDD_EINVAL;
    }
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    if (g->slab) {
        set_error("a sharded gauge field is solved collectively with qdd_solve, not queued");
        return QDD_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->g = g;
    r->bn = (size_t)g->hg.V * 24 * p->nrhs;
    r->b.reset(new (std::nothrow) double[r->bn]);
    if (!r->b) {
        set_error("no host memory for a copy of the sources (%zu bytes)", r->bn * sizeof(double));
        return QDD_ENOMEM;
    }
    par_copy(r->b.get(), b, r->bn);
    r->x = x;
    r->p = *p;
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        r->ticket = ctx->next_ticket++;
        *ticket = r->ticket;
        ctx->tickets[r->ticket] = r;
        ctx->queue.push_back(r);
        if (ctx->workers.empty())
            for (int k = 0; k < ctx->max_slots; k++) ctx->workers.emplace_back(worker_main, (Ctx *)ctx);
    }
    ctx->q_cv.notify_one();
    return QDD_OK;
}

qdd_status qdd_poll(qdd_ctx *ctx, uint64_t ticket, qdd_report *rep, double timeout_s)
{
    clear_error();
    if (!ctx) return QDD_EINVAL;
    static thread_local std::vector<double> hist;
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return QDD_EINVAL;
    }
    std::shared_ptr<Request> r = it->second;
    auto deadline = std::chrono::steady_clock::now() +
                    std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                        std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    while (!r->done) {
        if (ctx->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return QDD_ENOTREADY;
    }
    ctx->tickets.erase(it);
    if (rep) {
        *rep = r->rep;
        hist = r->hist;
        rep->res_history = hist.data();
        rep->n_history = (int)hist.size();
    }
    if (r->status != QDD_OK) set_error("%s", r->err.c_str());
    return r->status;
}

void qdd_destroy(qdd_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    delete ctx;
}

}  // extern "C"
