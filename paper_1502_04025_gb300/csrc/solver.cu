// Flexible GMRES(m), right-preconditioned by the Schwarz alternating procedure
// (arXiv:1502.04025, Sec. 3.1: flexible GMRES outer solver, multiplicative
// Schwarz preconditioner; the deflated restarts of the paper's solver are not
// part of this form).
//
//   x = 0; repeat:
//     r = b - D x (FP64, true residual); stop when |r| <= tol |b|
//     v_0 = r / |r|;  g = |r| e_0
//     for j = 0..m-1:
//       z_j = M_SAP v_j                          (preconditioner precision)
//       w   = D z_j                               (FP64, or FP32 on request)
//       h_ij = <v_i, w>, w -= sum h_ij v_i        (classical Gram-Schmidt, FP64,
//                                                  re-orthogonalised when |w| drops
//                                                  below |w_0|/sqrt(2), or always)
//       h_{j+1,j} = |w|;  v_{j+1} = w / h_{j+1,j}
//       Givens rotations on the host; |g_{j+1}| / |b| is the residual estimate
//     y = R^{-1} g;  x += sum y_j z_j (FP64)
//
// Right-hand sides are solved in lockstep: every kernel of a step handles all
// of them (the Schwarz kernel reuses each staged domain for every source), the
// Krylov algebra and the Hessenberg matrices are per right-hand side.  The
// only host round trip per step is one copy of the Gram-Schmidt coefficients
// and norms of all right-hand sides.
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qdd {

typedef std::complex<double> zc;

static size_t ebytes(qdd_prec p) { return p == QDD_PREC_F64 ? 16 : (p == QDD_PREC_F32 ? 8 : 4); }

// device scalar area (double2 units): dots1, dots2 [nrhs][m+2], norms1, norms2,
// bnorm [nrhs], coef [nrhs][m+1]
struct ScalarMap {
    int m, B;
    size_t dots1() const { return 0; }
    size_t dots2() const { return (size_t)B * (m + 2); }
    size_t nrm1() const { return 2 * (size_t)B * (m + 2); }
    size_t nrm2() const { return nrm1() + B; }
    size_t bnrm() const { return nrm2() + B; }
    size_t coef() const { return bnrm() + B; }
    size_t total() const { return coef() + (size_t)B * (m + 1); }
};

std::unique_ptr<Workspace> make_workspace() { return std::unique_ptr<Workspace>(new Workspace()); }

size_t workspace_bytes(const Gauge *g, int m, int B, qdd_prec sp, bool use_sap)
{
    const size_t V = g->hg.V, n = V * 12;
    const qdd_prec zp = sp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    size_t b = n * 16 * B * (size_t)(3 + m + 1) + n * ebytes(zp) * B * (size_t)m;
    if (use_sap) {
        b += 2 * n * ebytes(sp) * B;
        if (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S) b += 2 * V * 4 * B;
    }
    return b + (1 << 20);
}

size_t workspace_held(const Workspace *w)
{
    const DevMem *all[] = {&w->io, &w->b, &w->x, &w->V, &w->Z, &w->rho, &w->rho_s, &w->delta, &w->delta_s,
                           &w->dev, &w->scratch, &w->err};
    size_t t = 0;
    for (auto *d : all) t += d->bytes;
    return t;
}

void workspace_release(Workspace *w)
{
    DevMem *all[] = {&w->io, &w->b, &w->x, &w->V, &w->Z, &w->rho, &w->rho_s, &w->delta, &w->delta_s,
                     &w->dev, &w->scratch, &w->err};
    for (auto *d : all) d->release();
}

static qdd_status ensure_ws(Gauge *g, Workspace &w, int m, int B, qdd_prec sp, bool use_sap)
{
    Ctx *c = g->ctx;
    const size_t V = g->hg.V, n = V * 12;
    const qdd_prec zp = sp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    QDD_TRY(w.io.ensure(c, n * 16 * B));
    QDD_TRY(w.b.ensure(c, n * 16 * B));
    QDD_TRY(w.x.ensure(c, n * 16 * B));
    QDD_TRY(w.V.ensure(c, n * 16 * B * (size_t)(m + 1)));
    QDD_TRY(w.Z.ensure(c, n * ebytes(zp) * B * (size_t)m));
    if (use_sap) {
        QDD_TRY(w.rho.ensure(c, n * ebytes(sp) * B));
        QDD_TRY(w.delta.ensure(c, n * ebytes(sp) * B));
        if (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S) {
            QDD_TRY(w.rho_s.ensure(c, V * 4 * B));
            QDD_TRY(w.delta_s.ensure(c, V * 4 * B));
        }
    }
    ScalarMap sm{m, B};
    QDD_TRY(w.dev.ensure(c, sm.total() * sizeof(double2)));
    QDD_TRY(w.scratch.ensure(c, blas_scratch_elems(c) * sizeof(double2)));
    QDD_TRY(w.err.ensure(c, sizeof(int)));
    if (w.host_elems < sm.total()) {
        if (w.host) cudaFreeHost(w.host);
        w.host = nullptr;
        QDD_CUDA(cudaMallocHost((void **)&w.host, sm.total() * sizeof(double2)));
        w.host_elems = sm.total();
    }
    w.nrhs = B;
    w.m = m;
    w.sp = sp;
    return QDD_OK;
}

qdd_status solve_impl(Gauge *g, Workspace *wsp, const double *b_in, double *x_out, int on_device,
                      const qdd_solve_params *p, qdd_report *rep, cudaStream_t s, std::vector<double> *rel_out)
{
    auto t0 = std::chrono::steady_clock::now();
    Ctx *ctx = g->ctx;
    const int m = p->restart_m, B = p->nrhs;
    if (m < 1 || m > 64 || B < 1 || B > 64 || !(p->tol > 0) || p->max_restarts < 0 || p->nmr < 0 || p->ncy < 1 ||
        p->sap_prec < QDD_PREC_F64 || p->sap_prec > QDD_PREC_BF16S ||
        (p->arnoldi_prec != QDD_PREC_F64 && p->arnoldi_prec != QDD_PREC_F32 && p->arnoldi_prec != QDD_PREC_DF64) ||
        p->reorth < 0 || p->reorth > 2) {
        set_error("invalid solve parameters");
        return QDD_EINVAL;
    }
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    const qdd_prec sp = p->sap_prec;
    const qdd_prec zp = sp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    if ((p->arnoldi_prec == QDD_PREC_F32 || p->relax_eta > 0) && zp != QDD_PREC_F32) {
        set_error("an FP32 Arnoldi operator needs a single-precision preconditioner output");
        return QDD_EINVAL;
    }
    if (!(p->relax_eta >= 0)) {
        set_error("relax_eta must be >= 0");
        return QDD_EINVAL;
    }
    Workspace &w = *wsp;
    QDD_TRY(ensure_ws(g, w, m, B, sp, p->use_sap != 0));
    if (p->use_sap) QDD_TRY(ensure_copy(g, sp, s));
    if (p->arnoldi_prec != QDD_PREC_F64) QDD_TRY(ensure_copy(g, p->arnoldi_prec, s));
    if (p->relax_eta > 0) QDD_TRY(ensure_copy(g, QDD_PREC_F32, s));
    const int64_t n = (int64_t)g->hg.V * 12;
    const int64_t ldV = n * B;  // stride between basis vectors of one rhs
    double2 *V = w.V.as<double2>();
    double2 *X = w.x.as<double2>(), *Bv = w.b.as<double2>();
    double2 *dev = w.dev.as<double2>(), *host = w.host, *scr = w.scratch.as<double2>();
    ScalarMap sm{m, B};
    const size_t zb = ebytes(zp);
    char *Z = w.Z.as<char>();
    long long launches0 = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->timer.mu);
        for (int c = 0; c < 4; c++) launches0 += ctx->timer.launches[c];
    }
    double ms0[3];
    for (int c = 0; c < 3; c++) ms0[c] = ctx->timer.ms[c];
    long long sap0 = ctx->timer.launches[K_SAP];

    // ---- inputs
    const double *bsrc = b_in;
    if (!on_device) {
        QDD_CUDA(cudaMemcpyAsync(w.io.p, b_in, (size_t)n * 16 * B, cudaMemcpyHostToDevice, s));
        bsrc = w.io.as<double>();
    }
    QDD_TRY(launch_spinor_in(g, bsrc, Bv, nullptr, QDD_PREC_F64, B, s));
    QDD_CUDA(cudaMemsetAsync(X, 0, (size_t)n * 16 * B, s));
    QDD_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), s));
    for (int r = 0; r < B; r++) QDD_TRY(blas_norm2(ctx, Bv + r * n, n, dev + sm.bnrm() + r, scr, s));
    QDD_CUDA(cudaMemcpyAsync(host + sm.bnrm(), dev + sm.bnrm(), B * sizeof(double2), cudaMemcpyDeviceToHost, s));
    QDD_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bnorm(B);
    for (int r = 0; r < B; r++) bnorm[r] = std::sqrt(host[sm.bnrm() + r].x);

    std::vector<char> active(B, 1);
    std::vector<double> rel(B, 0.0), est(B, 0.0);
    std::vector<std::vector<zc>> H(B, std::vector<zc>((size_t)(m + 1) * m)), gv(B, std::vector<zc>(m + 1));
    std::vector<std::vector<double>> cs(B, std::vector<double>(m));
    std::vector<std::vector<zc>> sn(B, std::vector<zc>(m));
    std::vector<int> kr(B, 0);
    w.hist.clear();
    int iters = 0, restarts = 0;
    bool converged = false;
    qdd_status status = QDD_OK;
    SapBuffers sb{w.rho.p, w.delta.p, nullptr, w.rho_s.as<float>(), w.delta_s.as<float>()};

    for (int cycle = 0;; cycle++) {
        // ---- true residual into V_0
        if (cycle == 0)
            QDD_CUDA(cudaMemcpyAsync(V, Bv, (size_t)n * 16 * B, cudaMemcpyDeviceToDevice, s));
        else
            QDD_TRY(launch_dslash(g, QDD_PREC_F64, QDD_PREC_F64, X, nullptr, QDD_PREC_F64, V, nullptr, QDD_PREC_F64,
                                  Bv, B, s));
        for (int r = 0; r < B; r++) QDD_TRY(blas_norm2(ctx, V + r * n, n, dev + sm.nrm1() + r, scr, s));
        QDD_CUDA(cudaMemcpyAsync(host + sm.nrm1(), dev + sm.nrm1(), B * sizeof(double2), cudaMemcpyDeviceToHost, s));
        QDD_CUDA(cudaStreamSynchronize(s));
        bool all = true;
        for (int r = 0; r < B; r++) {
            double beta = std::sqrt(host[sm.nrm1() + r].x);
            if (!std::isfinite(beta)) {
                set_error("non-finite residual norm (rhs %d)", r);
                status = QDD_ENAN;
            }
            rel[r] = bnorm[r] > 0 ? beta / bnorm[r] : 0.0;
            if (rel[r] <= p->tol) active[r] = 0;
            all = all && !active[r];
            gv[r].assign(m + 1, zc(0, 0));
            gv[r][0] = beta;
            kr[r] = 0;
        }
        if (cycle > 0) w.hist.push_back(rel[0]);
        if (status != QDD_OK) break;
        if (all) {
            converged = true;
            break;
        }
        if (cycle > p->max_restarts) break;
        for (int r = 0; r < B; r++) QDD_TRY(blas_scale_by_norm(ctx, V + r * n, n, dev + sm.nrm1() + r, V + r * n, s));
        for (int r = 0; r < B; r++) std::fill(H[r].begin(), H[r].end(), zc(0, 0));

        std::vector<char> open(active);  // still iterating in this cycle
        int kmax = 0;
        for (int j = 0; j < m; j++) {
            double2 *vj = V + (int64_t)j * ldV;
            double2 *wv = V + (int64_t)(j + 1) * ldV;
            char *zj = Z + (size_t)j * n * B * zb;
            // z_j = M v_j
            if (p->use_sap) {
                QDD_TRY(launch_spinor_convert(g, vj, nullptr, QDD_PREC_F64, w.rho.p, w.rho_s.as<float>(), sp, B, s));
                sb.psi = zj;
                SeqScope seq(ctx->timer, K_SAP, s);
                for (int hs = 0; hs < 2 * p->ncy; hs++)
                    QDD_TRY(launch_sap_halfsweep(g, sp, sb, hs & 1, p->nmr, B, hs < 2, hs >= 1, 0, w.err.as<int>(), s,
                                                 hs >= 1, false));
            } else {
                QDD_TRY(launch_spinor_convert(g, vj, nullptr, QDD_PREC_F64, zj, nullptr, zp, B, s));
            }
            // w = D z_j; relaxed to FP32 once the residual is small enough
            // that the operator's error no longer limits the attainable
            // accuracy (inexact Krylov: error allowed ~ tol / residual)
            double est_now = 0;
            for (int r = 0; r < B; r++)
                if (open[r]) est_now = std::max(est_now, j == 0 ? rel[r] : est[r]);
            const bool relaxed = p->relax_eta > 0 && p->relax_eta * est_now <= 0.1 * p->tol;
            if (relaxed)
                QDD_TRY(launch_dslash(g, QDD_PREC_F32, QDD_PREC_F32, zj, nullptr, QDD_PREC_F32, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            else if (p->arnoldi_prec == QDD_PREC_F64 || p->arnoldi_prec == QDD_PREC_DF64)
                QDD_TRY(launch_dslash(g, p->arnoldi_prec, p->arnoldi_prec, zj, nullptr, zp, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            else
                QDD_TRY(launch_dslash(g, QDD_PREC_F32, QDD_PREC_F32, zj, nullptr, QDD_PREC_F32, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            // classical Gram-Schmidt, pass 1 (dots include <w, w>)
            for (int r = 0; r < B; r++) {
                if (!open[r]) continue;
                double2 *d1 = dev + sm.dots1() + (size_t)r * (m + 2);
                QDD_TRY(blas_cdot_multi(ctx, V + r * n, j + 2, ldV, wv + r * n, n, d1, scr, s));
                QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d1, wv + r * n, n, dev + sm.nrm1() + r,
                                              scr, s));
            }
            std::vector<char> two(B, 0);
            if (p->reorth == 2) {
                for (int r = 0; r < B; r++) {
                    if (!open[r]) continue;
                    double2 *d2 = dev + sm.dots2() + (size_t)r * (m + 2);
                    QDD_TRY(blas_cdot_multi(ctx, V + r * n, j + 1, ldV, wv + r * n, n, d2, scr, s));
                    QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d2, wv + r * n, n,
                                                  dev + sm.nrm2() + r, scr, s));
                    two[r] = 1;
                }
            }
            QDD_CUDA(cudaMemcpyAsync(host, dev, sm.coef() * sizeof(double2), cudaMemcpyDeviceToHost, s));
            QDD_CUDA(cudaStreamSynchronize(s));
            if (p->reorth == 1) {
                bool any = false;
                for (int r = 0; r < B; r++) {
                    if (!open[r]) continue;
                    double before = host[sm.dots1() + (size_t)r * (m + 2) + j + 1].x;  // <w,w> before projection
                    double after = host[sm.nrm1() + r].x;
                    if (after < 0.5 * before) {
                        two[r] = 1;
                        any = true;
                        double2 *d2 = dev + sm.dots2() + (size_t)r * (m + 2);
                        QDD_TRY(blas_cdot_multi(ctx, V + r * n, j + 1, ldV, wv + r * n, n, d2, scr, s));
                        QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d2, wv + r * n, n,
                                                      dev + sm.nrm2() + r, scr, s));
                    }
                }
                if (any) {
                    QDD_CUDA(cudaMemcpyAsync(host, dev, sm.coef() * sizeof(double2), cudaMemcpyDeviceToHost, s));
                    QDD_CUDA(cudaStreamSynchronize(s));
                }
            }
            iters++;
            bool all_done = true;
            for (int r = 0; r < B; r++) {
                if (!open[r]) continue;
                std::vector<zc> &h = H[r];
                for (int i = 0; i <= j; i++) {
                    double2 a = host[sm.dots1() + (size_t)r * (m + 2) + i];
                    zc hij(a.x, a.y);
                    if (two[r]) {
                        double2 c2 = host[sm.dots2() + (size_t)r * (m + 2) + i];
                        hij += zc(c2.x, c2.y);
                    }
                    h[(size_t)i * m + j] = hij;
                }
                double nn = two[r] ? host[sm.nrm2() + r].x : host[sm.nrm1() + r].x;
                double hn = std::sqrt(nn);
                if (!std::isfinite(hn)) {
                    set_error("non-finite Arnoldi norm (rhs %d, step %d)", r, j);
                    status = QDD_ENAN;
                }
                h[(size_t)(j + 1) * m + j] = hn;
                // v_{j+1} = w / h_{j+1,j}
                QDD_TRY(blas_scale_by_norm(ctx, wv + r * n, n, dev + (two[r] ? sm.nrm2() : sm.nrm1()) + r, wv + r * n,
                                           s));
                // rotations
                for (int i = 0; i < j; i++) {
                    zc a = h[(size_t)i * m + j], c2 = h[(size_t)(i + 1) * m + j];
                    h[(size_t)i * m + j] = cs[r][i] * a + sn[r][i] * c2;
                    h[(size_t)(i + 1) * m + j] = -std::conj(sn[r][i]) * a + cs[r][i] * c2;
                }
                zc a = h[(size_t)j * m + j], bb = h[(size_t)(j + 1) * m + j];
                double nu = std::sqrt(std::norm(a) + std::norm(bb));
                if (std::abs(a) == 0.0) {
                    cs[r][j] = 0.0;
                    sn[r][j] = 1.0;
                    h[(size_t)j * m + j] = bb;
                } else {
                    zc ph = a / std::abs(a);
                    cs[r][j] = std::abs(a) / nu;
                    sn[r][j] = ph * std::conj(bb) / nu;
                    h[(size_t)j * m + j] = ph * nu;
                }
                h[(size_t)(j + 1) * m + j] = 0;
                gv[r][j + 1] = -std::conj(sn[r][j]) * gv[r][j];
                gv[r][j] = cs[r][j] * gv[r][j];
                kr[r] = j + 1;
                est[r] = bnorm[r] > 0 ? std::abs(gv[r][j + 1]) / bnorm[r] : 0.0;
                if (r == 0) w.hist.push_back(est[0]);
                if (est[r] <= p->tol || hn == 0.0) open[r] = 0;
                all_done = all_done && !open[r];
            }
            kmax = j + 1;
            if (status != QDD_OK || all_done) break;
        }
        if (status != QDD_OK) break;
        // x += Z y per rhs
        for (int r = 0; r < B; r++) {
            if (!active[r] || kr[r] == 0) continue;
            int k = kr[r];
            std::vector<zc> y(k);
            const std::vector<zc> &h = H[r];
            for (int i = k - 1; i >= 0; i--) {
                zc acc = gv[r][i];
                for (int l = i + 1; l < k; l++) acc -= h[(size_t)i * m + l] * y[l];
                y[i] = acc / h[(size_t)i * m + i];
            }
            double2 *cf = host + sm.coef() + (size_t)r * (m + 1);
            for (int i = 0; i < k; i++) cf[i] = make_double2(y[i].real(), y[i].imag());
        }
        QDD_CUDA(cudaMemcpyAsync(dev + sm.coef(), host + sm.coef(), (size_t)B * (m + 1) * sizeof(double2),
                                 cudaMemcpyHostToDevice, s));
        for (int r = 0; r < B; r++) {
            if (!active[r] || kr[r] == 0) continue;
            QDD_TRY(blas_axpy_multi(ctx, Z + (size_t)r * n * zb, zp == QDD_PREC_F32, kr[r], n * B,
                                    dev + sm.coef() + (size_t)r * (m + 1), X + r * n, n, s));
        }
        (void)kmax;
        restarts = cycle;
    }

    // ---- output
    double *dst = on_device ? x_out : w.io.as<double>();
    QDD_TRY(launch_spinor_out(g, X, nullptr, dst, QDD_PREC_F64, B, s));
    if (!on_device) QDD_CUDA(cudaMemcpyAsync(x_out, w.io.p, (size_t)n * 16 * B, cudaMemcpyDeviceToHost, s));
    int derr = 0;
    QDD_CUDA(cudaMemcpyAsync(&host[sm.total() - 1], w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    QDD_CUDA(cudaStreamSynchronize(s));
    std::memcpy(&derr, &host[sm.total() - 1], sizeof(int));
    ctx->timer.resolve();
    if (derr && status == QDD_OK) {
        set_error("a bounded device wait ran out in the Schwarz kernel (flags %d)", derr);
        status = QDD_ETIMEOUT;
    }
    if (status == QDD_OK && !converged) {
        set_error("not converged after %d restarts (relative residual %.3e)", restarts, rel[0]);
        status = QDD_ENOCONV;
    }
    if (rel_out) *rel_out = rel;
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->converged = converged ? 1 : 0;
        rep->iters = iters;
        rep->restarts = restarts;
        double tr = 0, te = 0;
        for (int r = 0; r < B; r++) {
            tr = std::max(tr, rel[r]);
            te = std::max(te, est[r]);
        }
        rep->true_rel_res = tr;
        rep->est_rel_res = te;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(ctx->timer.mu);
        rep->ms_sap = ctx->timer.ms[K_SAP] - ms0[K_SAP];
        rep->ms_dslash = ctx->timer.ms[K_DSLASH] - ms0[K_DSLASH];
        rep->ms_blas = ctx->timer.ms[K_BLAS] - ms0[K_BLAS];
        rep->sap_launches = ctx->timer.launches[K_SAP] - sap0;
        long long l1 = 0;
        for (int c = 0; c < 4; c++) l1 += ctx->timer.launches[c];
        rep->kernel_launches = l1 - launches0;
        rep->n_history = (int)w.hist.size();
        rep->res_history = w.hist.data();
    }
    return status;
}

}  // namespace qdd
