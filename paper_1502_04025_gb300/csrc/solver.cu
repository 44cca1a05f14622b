// Flexible GMRES(m), right-preconditioned by the Schwarz alternating procedure,
// optionally with deflated restarts (arXiv:1502.04025, Sec. 3.1: the outer
// solver is flexible GMRES with deflated restarts, the preconditioner
// multiplicative Schwarz).
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
//       min |c - Hbar y| on the host (Householder QR); its norm / |b| is the
//       residual estimate
//     x += sum y_j z_j (FP64)
//   Deflated restart (dr_k = k > 0, after a full cycle): the k harmonic Ritz
//   vectors g of smallest modulus (eigenvectors of H_m + H_m^{-H} l^H l, l the
//   last row of Hbar) and the least-squares residual rho give an orthonormal
//   P_{k+1}; V_{k+1} <- V_{m+1} P_{k+1}, Z_k <- Z_m P_k (kept in FP64),
//   Hbar <- P_{k+1}^H Hbar P_k, c <- P_{k+1}^H rho, and the next cycle starts
//   at step k.  If the true residual has drifted from the implicit one the
//   restart falls back to the plain form.
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
#include "dense.h"

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

size_t workspace_bytes(const Gauge *g, int m, int B, qdd_prec sp, bool use_sap, int kdr)
{
    const size_t V = g->hg.V, n = V * 12;
    const qdd_prec zp = sp == QDD_PREC_F64 ? QDD_PREC_F64 : QDD_PREC_F32;
    size_t b = n * 16 * B * (size_t)(3 + m + 1) + n * ebytes(zp) * B * (size_t)m;
    if (use_sap) {
        b += n * ebytes(spinor_store(sp)) * B + sap_face_bytes(g->hg, sp, B);
        if (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S) b += V * 4 * B;
    }
    if (kdr > 0) b += n * 16 * B * (size_t)(3 * kdr + 1);
    return b + (1 << 20);
}

size_t workspace_held(const Workspace *w)
{
    const DevMem *all[] = {&w->io, &w->b, &w->x, &w->V, &w->Z, &w->rho, &w->rho_s, &w->face,
                           &w->dev, &w->scratch, &w->err, &w->ZR, &w->Vt, &w->ZRt, &w->P};
    size_t t = 0;
    for (auto *d : all) t += d->bytes;
    return t;
}

void workspace_release(Workspace *w)
{
    DevMem *all[] = {&w->io, &w->b, &w->x, &w->V, &w->Z, &w->rho, &w->rho_s, &w->face,
                     &w->dev, &w->scratch, &w->err, &w->ZR, &w->Vt, &w->ZRt, &w->P};
    for (auto *d : all) d->release();
}

static qdd_status ensure_ws(Gauge *g, Workspace &w, int m, int B, qdd_prec sp, bool use_sap, int kdr)
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
        QDD_TRY(w.rho.ensure(c, n * ebytes(spinor_store(sp)) * B));
        QDD_TRY(w.face.ensure(c, sap_face_bytes(g->hg, sp, B)));
        if (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S) QDD_TRY(w.rho_s.ensure(c, V * 4 * B));
    }
    if (kdr > 0) {
        QDD_TRY(w.ZR.ensure(c, n * 16 * B * (size_t)kdr));
        QDD_TRY(w.ZRt.ensure(c, n * 16 * B * (size_t)kdr));
        QDD_TRY(w.Vt.ensure(c, n * 16 * B * (size_t)(kdr + 1)));
        QDD_TRY(w.P.ensure(c, sizeof(double2) * B * (size_t)(m + 1) * (kdr + 1)));
    }
    ScalarMap sm{m, B};
    QDD_TRY(w.dev.ensure(c, sm.total() * sizeof(double2)));
    QDD_TRY(blas_scratch_ensure(c, w.scratch));
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

qdd_status solve_prepare(Gauge *g, Workspace *w, const qdd_solve_params *p, cudaStream_t s)
{
    const qdd_prec sp = p->use_sap == 2 ? mg_smoother_prec(g) : p->sap_prec;
    QDD_TRY(ensure_ws(g, *w, p->restart_m, p->nrhs, sp, p->use_sap == 1, p->dr_k));
    if (p->use_sap) QDD_TRY(ensure_copy(g, sp, s));
    if (p->arnoldi_prec != QDD_PREC_F64) QDD_TRY(ensure_copy(g, p->arnoldi_prec, s));
    if (p->relax_eta > 0 || p->arnoldi_prec == QDD_PREC_F32) {
        QDD_TRY(ensure_copy(g, QDD_PREC_F32, s));
        if (g->two_rows) QDD_TRY(ensure_links12(g, QDD_PREC_F32, s));
    }
    return QDD_OK;
}

qdd_status solve_impl(Gauge *g, Workspace *wsp, const double *b_in, double *x_out, int on_device,
                      const qdd_solve_params *p, qdd_report *rep, cudaStream_t s, std::vector<double> *rel_out)
{
    auto t0 = std::chrono::steady_clock::now();
    Ctx *ctx = g->ctx;
    const int m = p->restart_m, B = p->nrhs;
    if (m < 1 || m > 64 || B < 1 || B > 64 || !(p->tol > 0) || p->max_restarts < 0 || p->nmr < 0 || p->ncy < 1 ||
        !is_sap_prec(p->sap_prec) ||
        (p->arnoldi_prec != QDD_PREC_F64 && p->arnoldi_prec != QDD_PREC_F32 && p->arnoldi_prec != QDD_PREC_DF64) ||
        p->reorth < 0 || p->reorth > 2 || p->dr_k < 0 || p->dr_k >= m || p->use_sap < 0 || p->use_sap > 2) {
        set_error("invalid solve parameters");
        return QDD_EINVAL;
    }
    if (p->use_sap == 2 && (!g->mg || B != 1)) {
        set_error(g->mg ? "the multigrid preconditioner takes one right-hand side"
                        : "qdd_mg_setup has not been called");
        return QDD_EINVAL;
    }
    if (!g->have_clover) {
        set_error("set_clover has not been called");
        return QDD_EINVAL;
    }
    if (g->slab && (p->use_sap == 2 || p->dr_k > 0)) {
        set_error("a sharded gauge field solves with the Schwarz preconditioner or none, without deflation");
        return QDD_EINVAL;
    }
    const bool sharded = g->slab != nullptr;
    // the preconditioner's storage (the multigrid smoother's, when it is used)
    const qdd_prec sp = p->use_sap == 2 ? mg_smoother_prec(g) : p->sap_prec;
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
    QDD_TRY(solve_prepare(g, wsp, p, s));
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
    QDD_TRY(slab_allreduce(g, (double *)(host + sm.bnrm()), 2 * (size_t)B));  // sharded: over the ranks
    std::vector<double> bnorm(B);
    for (int r = 0; r < B; r++) bnorm[r] = std::sqrt(host[sm.bnrm() + r].x);

    std::vector<char> active(B, 1);
    std::vector<double> rel(B, 0.0), est(B, 0.0);
    // per rhs: Hbar (m+1) x m, right-hand side c of the small least-squares
    // problem, the columns of this cycle, the recycled count j0
    std::vector<dense::Mat> H(B, dense::Mat(m + 1, m));
    std::vector<std::vector<zc>> cv(B, std::vector<zc>(m + 1)), rho(B);
    std::vector<int> kr(B, 0);
    int j0 = 0;                  // columns carried over by a deflated restart (same for all rhs)
    bool pending_dr = false;     // the previous cycle ended ready for a deflated restart
    // FP32 Schwarz input: written by the scaling that makes v_j, which saves a
    // conversion pass per step (rho_ready: rho holds v_j of every right-hand side)
    float2 *rho32 = (p->use_sap == 1 && spinor_store(sp) == QDD_PREC_F32) ? w.rho.as<float2>() : nullptr;
    // 16-bit storage: the scaling writes the Schwarz input with its scales too
    const bool rho16 = p->use_sap == 1 && (sp == QDD_PREC_F16S || sp == QDD_PREC_BF16S);
    auto scale_v = [&](const double2 *src, int r, const double2 *nrm, double2 *dst) -> qdd_status {
        if (rho16)
            return launch_scale_convert(g, src, nrm, dst, (char *)w.rho.p + (size_t)r * n * 4,
                                        w.rho_s.as<float>() + (size_t)r * g->hg.V, sp, s);
        return blas_scale_by_norm(ctx, src, n, nrm, dst, s, rho32 ? rho32 + r * n : nullptr);
    };
    bool rho_ready = false;
    const int kdr = p->dr_k;
    w.hist.clear();
    int iters = 0, restarts = 0, deflated = 0;
    bool converged = false;
    qdd_status status = QDD_OK;
    SapBuffers sb{w.rho.p, w.face.p, nullptr, w.rho_s.as<float>()};
    double2 *ZR = w.ZR.as<double2>();

    for (int cycle = 0;; cycle++) {
        // ---- true residual into V_0 (FP64)
        if (cycle == 0)
            QDD_CUDA(cudaMemcpyAsync(V, Bv, (size_t)n * 16 * B, cudaMemcpyDeviceToDevice, s));
        else {
            QDD_TRY(slab_dslash_begin(g, X, false, false, B, s));  // sharded: boundary planes
            QDD_TRY(launch_dslash(g, QDD_PREC_F64, QDD_PREC_F64, X, nullptr, QDD_PREC_F64, pending_dr ? w.Vt.as<double2>() : V,
                                  nullptr, QDD_PREC_F64, Bv, B, s));
            QDD_TRY(slab_dslash_end(g, V, true, B, s));
        }
        double2 *R0 = (cycle > 0 && pending_dr) ? w.Vt.as<double2>() : V;
        for (int r = 0; r < B; r++) QDD_TRY(blas_norm2(ctx, R0 + r * n, n, dev + sm.nrm1() + r, scr, s));
        QDD_TRY(slab_allreduce_dev(g, dev + sm.nrm1(), B, s));
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
        }
        if (cycle > 0) w.hist.push_back(rel[0]);
        if (status != QDD_OK) break;
        if (all) {
            converged = true;
            break;
        }
        if (cycle > p->max_restarts) break;

        // ---- deflated restart (harmonic Ritz vectors of the last cycle), else plain restart
        rho_ready = false;
        bool deflate = pending_dr;
        std::vector<dense::Mat> Pm(B);
        if (deflate) {
            for (int r = 0; r < B && deflate; r++) {
                if (!active[r]) continue;
                // the implicit residual must still describe the true one
                double implicit = dense::nrm(rho[r]);
                double truth = rel[r] * bnorm[r];
                if (!(truth <= 2.0 * implicit + 1e-300)) { deflate = false; break; }
                const dense::Mat &Hb = H[r];
                dense::Mat Hm(m, m), rhs(m, m);
                for (int i = 0; i < m; i++)
                    for (int jj = 0; jj < m; jj++) Hm(i, jj) = Hb(i, jj);
                // F = H_m + H_m^{-H} l^H l, l = last row of Hbar
                dense::Mat HmH(m, m);
                for (int i = 0; i < m; i++)
                    for (int jj = 0; jj < m; jj++) {
                        HmH(i, jj) = std::conj(Hm(jj, i));
                        rhs(i, jj) = std::conj(Hb(m, i)) * Hb(m, jj);
                    }
                if (!dense::solve(HmH, rhs)) { deflate = false; break; }
                dense::Mat F(m, m);
                for (size_t t = 0; t < F.a.size(); t++) F.a[t] = Hm.a[t] + rhs.a[t];
                std::vector<zc> theta;
                dense::Mat G;
                if (!dense::eig(F, theta, G)) { deflate = false; break; }
                std::vector<int> ord(m);
                for (int i = 0; i < m; i++) ord[i] = i;
                std::stable_sort(ord.begin(), ord.end(),
                                 [&](int x, int y) { return std::abs(theta[x]) < std::abs(theta[y]); });
                dense::Mat Gk(m + 1, kdr);
                for (int c = 0; c < kdr; c++)
                    for (int i = 0; i < m; i++) Gk(i, c) = G(i, ord[c]);
                dense::Mat Q = dense::orthonormal(Gk);
                // last column: the least-squares residual, orthogonalised twice
                dense::Mat P(m + 1, kdr + 1);
                for (int i = 0; i <= m; i++)
                    for (int c = 0; c < kdr; c++) P(i, c) = Q(i, c);
                std::vector<zc> q = rho[r];
                for (int pass = 0; pass < 2; pass++)
                    for (int c = 0; c < kdr; c++) {
                        zc sc = 0;
                        for (int i = 0; i <= m; i++) sc += std::conj(Q(i, c)) * q[i];
                        for (int i = 0; i <= m; i++) q[i] -= sc * Q(i, c);
                    }
                double qn = dense::nrm(q);
                if (!(qn > 0)) { deflate = false; break; }
                for (int i = 0; i <= m; i++) P(i, kdr) = q[i] / qn;
                Pm[r] = P;
            }
        }
        if (deflate) {
            // upload P (row-major (m+1) x (kdr+1) per rhs), recombine V and Z on the device
            double2 *Pd = w.P.as<double2>();
            std::vector<double2> ph((size_t)B * (m + 1) * (kdr + 1), make_double2(0, 0));
            for (int r = 0; r < B; r++) {
                if (!active[r]) continue;
                for (int i = 0; i <= m; i++)
                    for (int c = 0; c <= kdr; c++) {
                        zc v = Pm[r](i, c);
                        ph[((size_t)r * (m + 1) + i) * (kdr + 1) + c] = make_double2(v.real(), v.imag());
                    }
            }
            QDD_CUDA(cudaMemcpyAsync(Pd, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
            double2 *Vt = w.Vt.as<double2>(), *ZRt = w.ZRt.as<double2>();
            for (int r = 0; r < B; r++) {
                if (!active[r]) continue;
                const double2 *Pr = Pd + (size_t)r * (m + 1) * (kdr + 1);
                // V_new[c] = sum_{i<=m} V_i P[i][c], c <= kdr
                QDD_TRY(blas_combine(ctx, V + r * n, false, m + 1, ldV, Pr, kdr + 1, kdr + 1, Vt + r * n, n * B, n,
                                     0, s));
                // Z_new[c] = sum_{i<j0} ZR_i P[i][c] + sum_{i=j0..m-1} Z_i P[i][c], c < kdr
                if (j0 > 0)
                    QDD_TRY(blas_combine(ctx, ZR + r * n, false, j0, ldV, Pr, kdr + 1, kdr, ZRt + r * n, n * B, n, 0,
                                         s));
                QDD_TRY(blas_combine(ctx, Z + ((size_t)j0 * n * B + r * n) * zb, zp == QDD_PREC_F32, m - j0,
                                     (int64_t)n * B, Pr + (size_t)j0 * (kdr + 1), kdr + 1, kdr, ZRt + r * n, n * B, n,
                                     j0 > 0 ? 1 : 0, s));
            }
            QDD_CUDA(cudaMemcpyAsync(V, Vt, (size_t)(kdr + 1) * n * 16 * B, cudaMemcpyDeviceToDevice, s));
            QDD_CUDA(cudaMemcpyAsync(ZR, ZRt, (size_t)kdr * n * 16 * B, cudaMemcpyDeviceToDevice, s));
            for (int r = 0; r < B; r++) {
                if (!active[r]) continue;
                const dense::Mat &P = Pm[r];
                dense::Mat Hn(m + 1, m);
                std::vector<zc> cn(m + 1, zc(0, 0));
                // Hbar_new = P^H Hbar P_k ; c_new = P^H rho
                for (int a2 = 0; a2 <= kdr; a2++) {
                    for (int b2 = 0; b2 < kdr; b2++) {
                        zc sum = 0;
                        for (int i = 0; i <= m; i++)
                            for (int jj = 0; jj < m; jj++)
                                sum += std::conj(P(i, a2)) * H[r](i, jj) * P(jj, b2);
                        Hn(a2, b2) = sum;
                    }
                    zc sum = 0;
                    for (int i = 0; i <= m; i++) sum += std::conj(P(i, a2)) * rho[r][i];
                    cn[a2] = sum;
                }
                H[r] = Hn;
                cv[r] = cn;
                kr[r] = kdr;
            }
            j0 = kdr;
            restarts++;
            deflated++;
        } else {
            for (int r = 0; r < B; r++) QDD_TRY(scale_v(R0 + r * n, r, dev + sm.nrm1() + r, V + r * n));
            rho_ready = rho32 != nullptr || rho16;
            for (int r = 0; r < B; r++) {
                H[r] = dense::Mat(m + 1, m);
                cv[r].assign(m + 1, zc(0, 0));
                cv[r][0] = rel[r] * bnorm[r];
                kr[r] = 0;
            }
            if (cycle > 0) restarts++;
            j0 = 0;
        }
        pending_dr = false;

        std::vector<char> open(active);  // still iterating in this cycle
        for (int j = j0; j < m; j++) {
            double2 *vj = V + (int64_t)j * ldV;
            double2 *wv = V + (int64_t)(j + 1) * ldV;
            char *zj = Z + (size_t)j * n * B * zb;
            // z_j = M v_j
            if (p->use_sap == 2) {
                QDD_TRY(mg_vcycle(g, vj, zj, zp, s));
            } else if (p->use_sap) {
                if (!rho_ready)
                    QDD_TRY(launch_spinor_convert(g, vj, nullptr, QDD_PREC_F64, w.rho.p, w.rho_s.as<float>(),
                                                  spinor_store(sp), B, s));
                rho_ready = false;
                sb.psi = zj;
                SeqScope seq(ctx->timer, K_SAP, s);
                for (int hs = 0; hs < 2 * p->ncy; hs++) {
                    // sharded: the face slots crossing the slab boundaries move
                    // while the interior domains are swept
                    if (sharded)
                        QDD_TRY(slab_sap_halfsweep(g, sp, sb, hs & 1, p->nmr, B, hs < 2, hs >= 1, w.err.as<int>(), s,
                                                   hs + 1 < 2 * p->ncy));
                    else
                        QDD_TRY(launch_sap_halfsweep(g, sp, sb, hs & 1, p->nmr, B, hs < 2, hs >= 1, 0,
                                                     w.err.as<int>(), s, hs >= 1, false));
                }
            } else {
                QDD_TRY(launch_spinor_convert(g, vj, nullptr, QDD_PREC_F64, zj, nullptr, zp, B, s));
            }
            // w = D z_j; relaxed to FP32 once the residual is small enough
            // that the operator's error no longer limits the attainable
            // accuracy (inexact Krylov: error allowed ~ tol / residual)
            double est_now = 0;
            for (int r = 0; r < B; r++)
                if (open[r]) est_now = std::max(est_now, j == j0 ? rel[r] : est[r]);
            const bool relaxed = p->relax_eta > 0 && p->relax_eta * est_now <= 0.1 * p->tol;
            QDD_TRY(slab_dslash_begin(g, zj, zp == QDD_PREC_F32, false, B, s));  // sharded: boundary planes
            if (relaxed)
                QDD_TRY(launch_dslash(g, QDD_PREC_F32, QDD_PREC_F32, zj, nullptr, QDD_PREC_F32, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            else if (p->arnoldi_prec == QDD_PREC_F64 || p->arnoldi_prec == QDD_PREC_DF64)
                QDD_TRY(launch_dslash(g, p->arnoldi_prec, p->arnoldi_prec, zj, nullptr, zp, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            else
                QDD_TRY(launch_dslash(g, QDD_PREC_F32, QDD_PREC_F32, zj, nullptr, QDD_PREC_F32, wv, nullptr,
                                      QDD_PREC_F64, nullptr, B, s));
            QDD_TRY(slab_dslash_end(g, wv, false, B, s));
            // classical Gram-Schmidt, pass 1 (dots include <w, w>)
            for (int r = 0; r < B; r++) {
                if (!open[r]) continue;
                // <w, w> (the last dot) only feeds the selective re-orthogonalisation test
                double2 *d1 = dev + sm.dots1() + (size_t)r * (m + 2);
                const int nd = p->reorth == 1 ? j + 2 : j + 1;
                QDD_TRY(blas_cdot_multi(ctx, V + r * n, nd, ldV, wv + r * n, n, d1, scr, s));
                QDD_TRY(slab_allreduce_dev(g, d1, nd, s));  // sharded: sums over the ranks
                QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d1, wv + r * n, n, dev + sm.nrm1() + r,
                                              scr, s));
                QDD_TRY(slab_allreduce_dev(g, dev + sm.nrm1() + r, 1, s));
            }
            std::vector<char> two(B, 0);
            if (p->reorth == 2) {
                for (int r = 0; r < B; r++) {
                    if (!open[r]) continue;
                    double2 *d2 = dev + sm.dots2() + (size_t)r * (m + 2);
                    QDD_TRY(blas_cdot_multi(ctx, V + r * n, j + 1, ldV, wv + r * n, n, d2, scr, s));
                    QDD_TRY(slab_allreduce_dev(g, d2, j + 1, s));
                    QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d2, wv + r * n, n,
                                                  dev + sm.nrm2() + r, scr, s));
                    QDD_TRY(slab_allreduce_dev(g, dev + sm.nrm2() + r, 1, s));
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
                        QDD_TRY(slab_allreduce_dev(g, d2, j + 1, s));
                        QDD_TRY(blas_caxpy_multi_norm(ctx, V + r * n, j + 1, ldV, d2, wv + r * n, n,
                                                      dev + sm.nrm2() + r, scr, s));
                        QDD_TRY(slab_allreduce_dev(g, dev + sm.nrm2() + r, 1, s));
                    }
                }
                if (any) {
                    QDD_CUDA(cudaMemcpyAsync(host, dev, sm.coef() * sizeof(double2), cudaMemcpyDeviceToHost, s));
                    QDD_CUDA(cudaStreamSynchronize(s));
                }
            }
            iters++;
            bool all_done = true;
            int scaled = 0;
            for (int r = 0; r < B; r++) {
                if (!open[r]) continue;
                scaled++;
                dense::Mat &h = H[r];
                for (int i = 0; i <= j; i++) {
                    double2 a = host[sm.dots1() + (size_t)r * (m + 2) + i];
                    zc hij(a.x, a.y);
                    if (two[r]) {
                        double2 c2 = host[sm.dots2() + (size_t)r * (m + 2) + i];
                        hij += zc(c2.x, c2.y);
                    }
                    h(i, j) = hij;
                }
                double nn = two[r] ? host[sm.nrm2() + r].x : host[sm.nrm1() + r].x;
                double hn = std::sqrt(nn);
                if (!std::isfinite(hn)) {
                    set_error("non-finite Arnoldi norm (rhs %d, step %d)", r, j);
                    status = QDD_ENAN;
                }
                h(j + 1, j) = hn;
                // v_{j+1} = w / h_{j+1,j}, with its FP32 copy for the next
                // preconditioner when every right-hand side goes on
                QDD_TRY(scale_v(wv + r * n, r, dev + (two[r] ? sm.nrm2() : sm.nrm1()) + r, wv + r * n));
                // residual estimate: min |c - Hbar y| over the j+1 columns
                dense::Mat Hs(j + 2, j + 1);
                for (int i = 0; i < j + 2; i++)
                    for (int l = 0; l < j + 1; l++) Hs(i, l) = h(i, l);
                std::vector<zc> cs(cv[r].begin(), cv[r].begin() + j + 2), y, res;
                dense::lstsq(Hs, cs, y, res);
                kr[r] = j + 1;
                est[r] = bnorm[r] > 0 ? dense::nrm(res) / bnorm[r] : 0.0;
                if (r == 0) w.hist.push_back(est[0]);
                if (est[r] <= p->tol || hn == 0.0) open[r] = 0;
                all_done = all_done && !open[r];
            }
            rho_ready = (rho32 != nullptr || rho16) && scaled == B;
            if (status != QDD_OK || all_done) break;
        }
        if (status != QDD_OK) break;
        // x += Z y per rhs (recycled z in FP64, the rest in the preconditioner's precision)
        bool full = true;
        for (int r = 0; r < B; r++) {
            if (!active[r] || kr[r] == 0) continue;
            int k = kr[r];
            dense::Mat Hs(k + 1, k);
            for (int i = 0; i <= k; i++)
                for (int l = 0; l < k; l++) Hs(i, l) = H[r](i, l);
            std::vector<zc> cs(cv[r].begin(), cv[r].begin() + k + 1), y;
            dense::lstsq(Hs, cs, y, rho[r]);
            rho[r].resize(m + 1, zc(0, 0));
            double2 *cf = host + sm.coef() + (size_t)r * (m + 1);
            for (int i = 0; i < k; i++) cf[i] = make_double2(y[i].real(), y[i].imag());
            full = full && k == m;
        }
        QDD_CUDA(cudaMemcpyAsync(dev + sm.coef(), host + sm.coef(), (size_t)B * (m + 1) * sizeof(double2),
                                 cudaMemcpyHostToDevice, s));
        for (int r = 0; r < B; r++) {
            if (!active[r] || kr[r] == 0) continue;
            const double2 *cf = dev + sm.coef() + (size_t)r * (m + 1);
            if (j0 > 0) QDD_TRY(blas_axpy_multi(ctx, ZR + r * n, false, j0, n * B, cf, X + r * n, n, s));
            QDD_TRY(blas_axpy_multi(ctx, Z + ((size_t)j0 * n * B + r * n) * zb, zp == QDD_PREC_F32, kr[r] - j0,
                                    n * B, cf + j0, X + r * n, n, s));
        }
        pending_dr = kdr > 0 && full;
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
        rep->deflated_restarts = deflated;
        rep->n_history = (int)w.hist.size();
        rep->res_history = w.hist.data();
    }
    return status;
}

}  // namespace qdd
