// Autotuner: domain shape and MR step count for a given lattice, precision
// and number of right-hand sides.
//
// The paper picks 4^4 or 8x4^3 domains so that a domain fits a core's cache
// (Sec. 3.3), finds 4-5 MR steps optimal for time-to-solution (Sec. 3.7) and
// models the load of N_d/2 independent domains on N_c cores as x/ceil(x)
// (Sec. 3.5).  On the GPU a domain is a CTA: the candidates are timed end to
// end (time-to-solution of the caller's solve, CUDA events), and each
// candidate's wave load x/ceil(x), with x = domains per colour / SMs, is
// reported beside its time.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

namespace qdd {

static void appendf(std::string &s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    s += buf;
}

}  // namespace qdd

using namespace qdd;

extern "C" qdd_status qdd_autotune(qdd_ctx *ctx, const int L[4], const double *links, int links_on_device,
                                   double c_sw, double kappa, const double *b, int b_on_device,
                                   const qdd_solve_params *p, const int *dom_candidates, int n_dom,
                                   const int *nmr_candidates, int n_nmr, qdd_tune_result *out, char *log,
                                   size_t log_len)
{
    clear_error();
    if (!ctx || !L || !links || !b || !p || !dom_candidates || n_dom < 1 || !out ||
        (n_nmr > 0 && !nmr_candidates)) {
        set_error("invalid argument");
        return QDD_EINVAL;
    }
    QDD_CUDA(cudaSetDevice(ctx->device));
    std::memset(out, 0, sizeof(*out));
    out->ms = -1;
    std::string js = "[";
    const size_t V = (size_t)L[0] * L[1] * L[2] * L[3];
    const size_t bbytes = V * 24 * sizeof(double) * (size_t)p->nrhs;
    // one device copy of b and one output buffer shared by all candidates
    DevMem bdev, xdev;
    const double *bd = b;
    if (!b_on_device) {
        QDD_TRY(bdev.alloc(ctx, bbytes));
        QDD_CUDA(cudaMemcpy(bdev.p, b, bbytes, cudaMemcpyHostToDevice));
        bd = bdev.as<double>();
    }
    QDD_TRY(xdev.alloc(ctx, bbytes));
    cudaStream_t st = nullptr;
    QDD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QDD_CUDA(cudaEventCreate(&e0));
    QDD_CUDA(cudaEventCreate(&e1));
    int tried = 0;
    bool first = true;
    for (int di = 0; di < n_dom; di++) {
        const int *dom = dom_candidates + 4 * di;
        qdd_gauge *g = nullptr;
        qdd_status s = qdd_create_gauge_field(ctx, L, dom, links, links_on_device, &g);
        if (s != QDD_OK) {
            appendf(js, "%s{\"dom\":[%d,%d,%d,%d],\"error\":\"%s\"}", first ? "" : ",", dom[0], dom[1], dom[2],
                    dom[3], qdd_last_error());
            first = false;
            continue;
        }
        s = qdd_set_clover(g, c_sw, kappa);
        if (s != QDD_OK) {
            qdd_destroy_gauge(g);
            cudaStreamDestroy(st);
            return s;
        }
        const double load = qdd_load_model(g->hg.Nd2, (double)ctx->nsm);
        const int nn = n_nmr > 0 ? n_nmr : 1;
        for (int k = 0; k < nn; k++) {
            qdd_solve_params q = *p;
            if (n_nmr > 0) q.nmr = nmr_candidates[k];
            qdd_report rep;
            // one untimed solve (buffers, copies), then one timed
            s = solve_impl(g, g->ws ? g->ws.get() : (g->ws = make_workspace()).get(), bd, xdev.as<double>(), 1, &q,
                           &rep, st);
            if (s != QDD_OK && s != QDD_ENOCONV) {
                qdd_destroy_gauge(g);
                cudaStreamDestroy(st);
                return s;
            }
            QDD_CUDA(cudaEventRecord(e0, st));
            s = solve_impl(g, g->ws.get(), bd, xdev.as<double>(), 1, &q, &rep, st);
            QDD_CUDA(cudaEventRecord(e1, st));
            QDD_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            QDD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            tried++;
            bool ok = (s == QDD_OK) && rep.converged;
            appendf(js,
                    "%s{\"dom\":[%d,%d,%d,%d],\"nmr\":%d,\"ms\":%.4f,\"iters\":%d,\"restarts\":%d,"
                    "\"converged\":%s,\"domains_per_colour\":%d,\"wave_load\":%.4f}",
                    first ? "" : ",", dom[0], dom[1], dom[2], dom[3], q.nmr, ms, rep.iters, rep.restarts,
                    ok ? "true" : "false", g->hg.Nd2, load);
            first = false;
            if (ok && (out->ms < 0 || ms < out->ms)) {
                out->ms = ms;
                std::memcpy(out->dom, dom, 4 * sizeof(int));
                out->nmr = q.nmr;
                out->iters = rep.iters;
                out->wave_load = load;
            }
        }
        qdd_destroy_gauge(g);
    }
    js += "]";
    out->n_tried = tried;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (log && log_len) {
        std::strncpy(log, js.c_str(), log_len - 1);
        log[log_len - 1] = 0;
    }
    if (out->ms < 0) {
        set_error("no candidate converged");
        return QDD_ENOCONV;
    }
    return QDD_OK;
}
