/*
 * qdd.h -- C ABI of libqdd, a GB300 (sm_103a) solver for the Wilson-clover
 * Dirac equation D x = b by flexible GMRES preconditioned with the Schwarz
 * alternating procedure (multiplicative Schwarz, "SAP") whose domain solver is
 * minimal-residual (MR) with even-odd preconditioning, as described in
 * arXiv:1502.04025, Sec. 3.1 ("Algorithm and implementation overview").
 *
 * Host layouts (every pointer argument named "host layout"):
 *   site index   n = x + Lx*(y + Ly*(z + Lz*t))  (x fastest), periodic lattice
 *   links        double complex U[n][mu][a][b], mu = 0..3 for x,y,z,t;
 *                U_mu(n) joins n to n+mu.  Re/Im interleaved, 18 doubles per link.
 *   spinors      double complex psi[n][s][c], s = 0..3 spin, c = 0..2 colour;
 *                24 doubles per site; nrhs spinors are stored back to back.
 * Conventions of the operator (the paper names it but prints no formula):
 *   D = A - kappa*H,
 *   H psi(n) = sum_mu (1-gamma_mu) U_mu(n) psi(n+mu) + (1+gamma_mu) U_mu(n-mu)^+ psi(n-mu),
 *   A(n) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(n),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F = traceless part of (Q - Q^+)/8,
 *   Q the four-leaf clover; gammas in the Hermitian chiral basis with
 *   gamma_5 = diag(1,1,-1,-1).
 *
 * Ownership: the caller owns every buffer it passes; the library owns the
 * objects it creates (context, gauge field, their device copies) until the
 * matching destroy call.  Pointers flagged "on_device" are CUDA device
 * pointers of the context's device; otherwise host pointers.  "stream" is a
 * cudaStream_t (NULL = the legacy default stream); every call returns only
 * after its results are in the caller's buffers.
 *
 * Errors: every call returns a qdd_status; QDD_OK is 0.  On failure the
 * thread-local message of qdd_last_error() says why.  No call aborts the
 * process.  A non-converged solve returns QDD_ENOCONV with x holding the best
 * iterate and the report filled in.
 */
#ifndef QDD_H
#define QDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qdd_ctx qdd_ctx;
typedef struct qdd_gauge qdd_gauge;

typedef enum {
    QDD_OK = 0,
    QDD_EINVAL = 1,   /* invalid argument (sizes, geometry, null pointer) */
    QDD_ENOMEM = 2,   /* device or host allocation failed */
    QDD_EBUDGET = 3,  /* the request would exceed the context's HBM budget */
    QDD_ENOCONV = 4,  /* solver stopped at max_restarts without reaching tol */
    QDD_ENAN = 5,     /* a NaN or Inf appeared in a residual */
    QDD_ETIMEOUT = 6, /* a bounded wait ran out (device flag or host poll) */
    QDD_ECUDA = 7,    /* a CUDA runtime call failed */
    QDD_ENOTREADY = 8, /* serving: the ticket is still in flight */
    QDD_ECOMM = 9      /* a communication hook of a sharded gauge field failed */
} qdd_status;

/* Precision of the Schwarz preconditioner (arithmetic / storage), and of the
 * operator inside the Arnoldi step.  The outer FGMRES vector algebra is
 * always FP64.  F16S / BF16S: FP32 arithmetic on 16-bit storage of links
 * (unscaled, |U_ab| <= 1), clover blocks and residual spinors (one FP32
 * scale per site, stored values in [-1, 1]); the paper stores links and
 * clover in half precision with single-precision spinors (Sec. 3.3). */
typedef enum {
    QDD_PREC_F64 = 0,
    QDD_PREC_F32 = 1,
    QDD_PREC_F16S = 2,
    QDD_PREC_BF16S = 3,
    QDD_PREC_DF64 = 4, /* operator only: FP64-class accuracy (about 2^-46) from
                          pairs of FP32 numbers; links and clover split into
                          hi + lo parts.  For qdd_apply_D and arnoldi_prec. */
    QDD_PREC_H16 = 5   /* the paper's half precision (Sec. 3.3): FP16 links and
                          clover (per-site scale), FP32 spinors, FP32 arithmetic */
} qdd_prec;

typedef struct {
    double tol;           /* stop when |b - D x| <= tol |b| (true FP64 residual) */
    int restart_m;        /* FGMRES cycle length m (<= 64) */
    int max_restarts;     /* restarts after the first cycle */
    int nmr;              /* MR steps per domain visit */
    int ncy;              /* Schwarz cycles per preconditioner application */
    qdd_prec sap_prec;    /* preconditioner precision */
    qdd_prec arnoldi_prec;/* QDD_PREC_F64, QDD_PREC_DF64 or QDD_PREC_F32: operator
                             in w = D z_j (the restart residual is always FP64) */
    int use_sap;          /* preconditioner: 0 none (plain GMRES), 1 the
                             Schwarz method (SAP), 2 the two-level multigrid
                             V-cycle with the Schwarz smoother (qdd_mg_setup
                             first; one right-hand side; its own smoother
                             parameters replace nmr, ncy and sap_prec) */
    int nrhs;             /* right-hand sides solved together (1..12) */
    int reorth;           /* Gram-Schmidt: 0 classical, 1 classical with
                             selective re-orthogonalisation, 2 twice always */
    double relax_eta;     /* relaxed Arnoldi operator (inexact Krylov): when
                             > 0, a step whose residual estimate est satisfies
                             relax_eta * est <= 0.1 * tol applies w = D z_j in
                             FP32 (relax_eta = the FP32 operator's relative
                             error, e.g. 1e-6); 0 = off.  Needs an FP32
                             preconditioner output.  Convergence is still
                             decided on the FP64 true residual. */
    int dr_k;             /* deflated restarts (Sec. 3.1: the outer solver is
                             flexible GMRES with deflated restarts): keep the
                             dr_k harmonic Ritz vectors of smallest modulus
                             across each restart (0 = plain restarts;
                             0 <= dr_k < restart_m). */
} qdd_solve_params;

typedef struct {
    int converged;          /* all right-hand sides reached tol */
    int iters;              /* Arnoldi steps (lockstep over right-hand sides) */
    int restarts;           /* restarts performed */
    double true_rel_res;    /* max over rhs of |b - D x| / |b| at return */
    double est_rel_res;     /* max over rhs of the last Givens estimate */
    double seconds;         /* host wall time of the call */
    double ms_sap;          /* device time in the Schwarz kernels (profiling on) */
    double ms_dslash;       /* device time in full-lattice operator kernels */
    double ms_blas;         /* device time in FP64 vector kernels */
    long long sap_launches; /* Schwarz block-kernel launches */
    long long kernel_launches; /* all kernel launches of the call */
    int deflated_restarts;  /* restarts that kept harmonic Ritz vectors (dr_k > 0) */
    int n_history;          /* entries of res_history */
    const double *res_history; /* estimated relative residual per iteration of
                                  rhs 0, and the true one at each restart;
                                  library-owned, valid until the next solve */
} qdd_report;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = 80% of the device's total memory);
 * allocations beyond it fail with QDD_EBUDGET. */
qdd_status qdd_create(qdd_ctx **ctx, int device, size_t hbm_budget_bytes);
void qdd_destroy(qdd_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *qdd_last_error(void);

/* Per-kernel-class device timing with CUDA events: classes is a bit mask of
 * QDD_PROF_* (0 = off); every launch of a selected class gets an event pair
 * on its stream.  Launch counts are kept for every class regardless.  Results
 * land in qdd_report's ms_* fields and in qdd_get_kernel_times. */
#define QDD_PROF_SAP 1
#define QDD_PROF_DSLASH 2
#define QDD_PROF_BLAS 4
#define QDD_PROF_OTHER 8
#define QDD_PROF_ALL 15
qdd_status qdd_set_profiling(qdd_ctx *ctx, int classes);

/* Kernel-class timings of the context since the last reset:
 * out[0..1] = (ms, launches) of SAP block kernels, out[2..3] of full-lattice
 * operator kernels, out[4..5] of FP64 vector kernels.  reset != 0 zeroes them. */
qdd_status qdd_get_kernel_times(qdd_ctx *ctx, double out[6], int reset);

/*
 * Measured arithmetic peak of device `device` (not part of the method: the
 * denominator of the rooflines of the ALU-bound steps).  Runs a chain of
 * independent fused multiply-adds on every SM, in FP64 (fp64 != 0) or FP32,
 * for about target_ms milliseconds (0 < target_ms <= 10000), timed with CUDA
 * events; *tflops = 2 flop per FMA / elapsed time, *ms (may be NULL) = the
 * elapsed time.  Synchronous; allocates and frees a small output buffer.
 */
qdd_status qdd_measure_fma_peak(int device, int fp64, double target_ms, double *tflops, double *ms);

/* Algorithmic work of the kernels launched since the last reset of
 * qdd_get_kernel_times: out[0..1] = (flop, bytes) of SAP block kernels,
 * out[2..3] of full-lattice operator kernels, out[4..5] of FP64 vector
 * kernels.  Only the FP64 vector kernels count theirs (8 flop per complex
 * multiply-add; 16 bytes per FP64 and 8 per FP32 complex element read or
 * written once); the other classes report 0. */
qdd_status qdd_get_kernel_work(qdd_ctx *ctx, double out[6]);

/* Bytes of device memory the context holds now, and its budget. */
qdd_status qdd_memory(qdd_ctx *ctx, size_t *used, size_t *budget);

/* ------------------------------------------------------------ gauge field */

/*
 * Upload a gauge field and fix its domain decomposition (Sec. 3.1: the
 * lattice is split into domains; Sec. 3.3: domains of 4^4 or 8x4^3 sites).
 * L[4]: lattice extents; dom[4]: domain extents.  Each dom[mu] must be even
 * and divide L[mu], and L[mu]/dom[mu] must be even (>= 2), so that the
 * two-colour checkerboard of domains is consistent; the product of dom must
 * be <= 512.  links: host layout, on the host or (links_on_device) the
 * device.  The device keeps FP64 links in a domain-blocked, parity-split,
 * plane-major layout, plus lower-precision copies made on demand.
 */
qdd_status qdd_create_gauge_field(qdd_ctx *ctx, const int L[4], const int dom[4], const double *links,
                                  int links_on_device, qdd_gauge **g);
void qdd_destroy_gauge(qdd_gauge *g);

/*
 * Two-row link storage for the full-lattice operator in FP32, FP16 and BF16
 * (not part of the paper, which stores whole links): an SU(3) link's third
 * row is the complex conjugate of the cross product of its first two (the
 * cofactors of a unitary matrix of determinant 1), so those operators read
 * 6 of the 9 entries and rebuild the rest, 96 of 288 bytes per site fewer in
 * FP32.  At creation every link is checked on the device (max |U U^+ - 1|
 * and |det U - 1| <= 1e-10); when all pass, two-row storage is on.
 * qdd_set_link_compression(g, 0) switches it off; (g, 1) switches it back
 * on and returns QDD_EINVAL for a field that failed the check.  The FP64
 * and double-float operators and the Schwarz kernel read whole links.
 * qdd_link_compression reports the setting and the check's outcome.
 */
qdd_status qdd_set_link_compression(qdd_gauge *g, int two_rows);
qdd_status qdd_link_compression(qdd_gauge *g, int *two_rows, int *is_su3);

/*
 * Form of the Schwarz block kernel.  3 runs two threads per even/odd site
 * pair, each with two of the four directions and one clover block (FP32
 * arithmetic, links and clover staged, half a domain a multiple of 32 sites,
 * at most 512 threads; otherwise the one-thread form of 0 runs); its partial
 * sums are added in another order, so it agrees with the one-thread form to
 * rounding.  0 (default) runs form 3 where it applies with FP32 links, and
 * otherwise one thread per site pair, staging the domain's links and, when
 * it fits, its clover in shared memory, with the domain size fixed at
 * compile time for 4^4 domains in 16-bit storage.  1 stages the links only,
 * reads the clover through the cache and is compiled for three CTAs per SM
 * (FP32 arithmetic on domains of at most 256 sites; otherwise 0 runs); 2 is
 * the one-thread form with the domain size always taken at run time.  Forms
 * 1 and 2 give the same bits as the one-thread form of 0.  The paper sizes
 * its domains to the cache (Sec. 3.3); on the GPU the choice trades staged
 * data and registers against the number of warps an SM holds.
 * Returns QDD_EINVAL for a null field or a form outside 0..3.
 */
qdd_status qdd_set_schwarz_variant(qdd_gauge *g, int variant);

/*
 * Range-checked build (test aid; compute-sanitizer stands in elsewhere).
 * A library built with -DQDD_CHECK (libqdd_check.so) tests the indices of
 * the Schwarz kernel's stencil, face-slot and reduction accesses, of the
 * full-lattice operators' neighbour reads and of the multigrid kernels'
 * neighbour-domain reads; one out of range is counted and
 * its access skipped.  *hits = the count since the library was loaded.  The
 * normal build sets *hits = 0 and returns QDD_EINVAL.
 */
qdd_status qdd_check_hits(unsigned long long *hits);

/*
 * Range-checked build only (test aid for the device-side failure path): the
 * poll limit of the Schwarz kernel's first bounded wait, the one for the
 * staging of a domain's links and clover, on device `device` (default
 * 1 << 22).  With 0 the wait gives up at once: the kernel sets its timeout
 * flag, waits (with its own fixed limit) until its staging copies have
 * landed, and returns, and the calling entry point reports QDD_ETIMEOUT.
 * Nothing spins without a limit.  The normal build returns QDD_EINVAL.
 */
qdd_status qdd_check_set_wait_limit(int device, unsigned spins);

/*
 * Build the clover term A = 1 + i kappa c_sw sum sigma F (two Hermitian 6x6
 * chirality blocks per site) and the inverse blocks on odd sites used by the
 * even-odd domain solver (Sec. 3.1, footnote on the domain inversion).  Must
 * be called before apply_D / sap_apply / solve; may be called again with new
 * (c_sw, kappa).  Returns QDD_EINVAL if a block is singular.
 */
qdd_status qdd_set_clover(qdd_gauge *g, double c_sw, double kappa);

/*
 * Clover blocks in the host site order: out[n][blk][i][j] complex (V*2*36
 * complex), blk 0 = spins {0,1}, blk 1 = spins {2,3}, index i = s*3 + c
 * within the block.  which = 0: A on every site; which = 1: the Schwarz form
 * (A on even sites, A^{-1} on odd sites).  out: host pointer.
 */
qdd_status qdd_get_clover(qdd_gauge *g, int which, double *out);

/* ------------------------------------------------------ sharded lattices */

/*
 * Communication hooks of a lattice sharded over ranks (Sec. 3.6 of the paper
 * distributes the lattice over processors and exchanges the boundaries).
 * The caller implements them with its own communication library; every rank
 * calls the collective entry points below in the same order.  Buffers are
 * host memory owned by the library for the duration of the call.
 *   allreduce_sum  buf[0..n) <- the sum over all ranks of buf[0..n) (doubles)
 *   shift          cyclic shift along the rank ring: send to_up (bytes) to
 *                  rank (rank+1) mod size and to_dn to (rank-1) mod size;
 *                  receive from (rank-1) mod size into from_dn and from
 *                  (rank+1) mod size into from_up (equal sizes everywhere;
 *                  with size 1 a rank is its own neighbour both ways)
 * Both return 0 on success; anything else aborts the call with QDD_ECOMM.
 */
typedef struct {
    void *user;  /* passed back to the hooks */
    int rank, size;
    int (*allreduce_sum)(void *user, double *buf, size_t n);
    int (*shift)(void *user, const void *to_up, void *from_dn, const void *to_dn, void *from_up, size_t bytes);
} qdd_comm;

/*
 * A gauge field sharded in the time direction (Sec. 3.6: the lattice is
 * split over processors, here into slabs of whole domains along t).  This
 * rank owns the local lattice Lloc = (Lx, Ly, Lz, lt) at global times
 * t0 .. t0+lt-1, with domains dom; lt/dom[3] must be even (>= 2) and t0 a
 * multiple of 2*dom[3], so that the domain colouring is the global one.
 * links_ext: the links of the extended local lattice (Lx, Ly, Lz,
 * lt + 2*dom[3]) in the host layout, its first plane at global time
 * t0 - dom[3] (periodic in the global lattice): the owned planes plus one
 * domain block of halo on each side, which the clover term of the boundary
 * planes needs.  comm: the rank's hooks (copied; `user` must stay valid
 * until the gauge field is destroyed).  Spinors of every entry point are in
 * the host layout of Lloc.  qdd_set_clover, qdd_apply_D (outputs F64, DF64,
 * F32), qdd_sap_apply and qdd_solve (use_sap 0 or 1, no deflation) then act
 * collectively: the Schwarz half-sweeps exchange the face slots that cross
 * the slab boundaries (a cyclic shift after every half-sweep), the operator
 * corrects its two boundary planes with the neighbours' hops, and the solver
 * sums its dot products and norms over the ranks.  Other entry points treat
 * the field as a periodic local lattice.
 */
qdd_status qdd_create_gauge_field_slab(qdd_ctx *ctx, const int Lloc[4], const int dom[4], const double *links_ext,
                                       int links_on_device, const qdd_comm *comm, qdd_gauge **g);

/*
 * Host-only: the face slots a sharded lattice exchanges after a half-sweep
 * of colour `colour` (the receiving domains have the other colour).
 * out[0..2] = (first domain slot, domain count, direction) of the region
 * sent to rank+1 (the first t-block's slots fed from below), out[3..5] the
 * same for the region sent to rank-1 (the last t-block's slots fed from
 * above); a direction's slots of domain d are face[d][k][foff[dir] ..
 * foff[dir] + Vd/dom[3]) for the six components k.
 */
qdd_status qdd_slab_regions(const int Lloc[4], const int dom[4], int colour, int out[6]);

/* Host-only: the face-slot layout of a domain shape: foff[8] the first slot
 * of each direction (k = 2*mu + 0 forward, 1 backward hop of the receiving
 * site), fcoord[Vd] the packed transverse index of each domain site (byte mu
 * = the index of its coordinates transverse to mu); either may be NULL. */
qdd_status qdd_layout_faces(const int L[4], const int dom[4], int foff[8], uint32_t *fcoord);

/* ------------------------------------------------------------- operators */

/*
 * out = D in for nrhs spinors (host layout), periodic boundary conditions.
 * prec = QDD_PREC_F64 computes in FP64; QDD_PREC_DF64 in double-float
 * (FP32 pairs, about 2^-46 relative); QDD_PREC_F32 converts links, clover
 * and input to FP32 and computes in FP32 (1848 flop per site); F16S / BF16S
 * read 16-bit links/clover/spinor with FP32 arithmetic.
 */
qdd_status qdd_apply_D(qdd_gauge *g, const double *in, double *out, int nrhs, qdd_prec prec, int on_device,
                       void *stream);

/*
 * One application of the Schwarz preconditioner psi = M eta (Sec. 3.1): zero
 * start, n_half colour half-sweeps (colour 0, 1, 0, ...; 2*ncy for ncy
 * cycles), each running nmr even-odd MR steps on every domain of the colour
 * with Dirichlet boundaries, then updating the residual of the neighbouring
 * domains.  rho (may be NULL) receives the maintained residual eta - D psi.
 * eta, psi, rho: host layout, nrhs spinors each.
 */
qdd_status qdd_sap_apply(qdd_gauge *g, const double *eta, double *psi, double *rho, int nrhs, int nmr, int n_half,
                         qdd_prec prec, int on_device, void *stream);

/* ----------------------------------------------------------------- solver */

/* Default parameters: tol 1e-10, m 16, 50 restarts, nmr 4, ncy 4, F32 SAP,
 * F64 Arnoldi operator, SAP on, 1 rhs, selective re-orthogonalisation,
 * no relaxation, no deflation. */
void qdd_default_params(qdd_solve_params *p);

/*
 * Solve D x = b (Sec. 3.1: flexible GMRES, right-preconditioned by SAP) for
 * p->nrhs right-hand sides in host layout.  x is an output (zero initial
 * guess).  Convergence is tested on the true FP64 residual recomputed at
 * every restart.  rep may be NULL.
 */
qdd_status qdd_solve(qdd_gauge *g, const double *b, double *x, int on_device, const qdd_solve_params *p,
                     qdd_report *rep, void *stream);

/* -------------------------------------------------------------- multigrid */

/*
 * Two-level aggregation multigrid preconditioner whose smoother is the
 * Schwarz method (Sec. 2.4 of the paper: the Krylov solver is preconditioned
 * by a V-cycle with the domain-decomposition preconditioner as smoother; the
 * paper gives no formula, the construction below is this library's reading).
 *   aggregates  the gauge field's Schwarz domains, each split by chirality
 *               (spins {0,1} and {2,3}), so the prolongator commutes with gamma5
 *   setup       the nv given vectors w_k are each replaced setup_iters times by
 *               M_SAP w_k (setup_ncy Schwarz cycles of nmr MR steps) and
 *               normalised; their restrictions to every aggregate-chirality
 *               block are orthonormalised (modified Gram-Schmidt, twice) and
 *               become the prolongator's columns P (stored in FP32)
 *   coarse      D_c = P^H D P, a 9-point stencil of (2 nv) x (2 nv) blocks on
 *               the lattice of domains (FP32)
 *   V-cycle     e ~ D_c^{-1} P^H v by one GMRES cycle of coarse_iters steps from
 *               zero (fewer on an exact breakdown), run on the device without
 *               host round trips, z = P e, then z += M_SAP(v - D z) with
 *               post_ncy Schwarz cycles
 *   bootstrap   the adaptive part of the setup, repeated `bootstrap` times:
 *               each w_k becomes the V-cycle of the method built so far
 *               applied to column k of P (as a fine field), normalised, and
 *               P and D_c are rebuilt from the new w_k
 */
typedef struct {
    int nv;            /* vectors per aggregate and chirality (1..16) */
    int setup_iters;   /* smoothing passes over the vectors */
    int setup_ncy;     /* Schwarz cycles per smoothing pass */
    int nmr;           /* MR steps per domain visit of the smoother */
    int post_ncy;      /* Schwarz cycles after the coarse correction (0 = none) */
    int coarse_iters;  /* steps of the coarse GMRES cycle (1..64) */
    qdd_prec sap_prec; /* the smoother's precision (as qdd_solve_params) */
    int bootstrap;     /* adaptive setup passes after the first build (0..8) */
} qdd_mg_params;

/* nv 8, setup_iters 3, setup_ncy 2, nmr 4, post_ncy 2, coarse_iters 12,
 * FP32 smoother, no bootstrap pass. */
void qdd_mg_default_params(qdd_mg_params *p);

/* Builds the preconditioner on g (replacing an earlier one).  w0: nv random
 * spinor fields in the host layout, nv*V*12 complex doubles (host or device
 * per on_device), read only.  The random numbers are the caller's, so that a
 * reference implementation can start from the same ones.  Holds
 * nv*V*96 bytes (P) plus the coarse operator and V-cycle work buffers until
 * the gauge field is destroyed.  QDD_EINVAL for bad parameters or before
 * qdd_set_clover. */
qdd_status qdd_mg_setup(qdd_gauge *g, const qdd_mg_params *p, const double *w0, int on_device);

/* z = M_MG v (one V-cycle) for one spinor in the host layout. */
qdd_status qdd_mg_vcycle(qdd_gauge *g, const double *v, double *z, int on_device, void *stream);

/* The prolongator's columns as nv spinor fields in the host layout (host
 * pointer, nv*V*12 complex doubles): field k holds column k of every
 * aggregate-chirality block. */
qdd_status qdd_mg_get_basis(qdd_gauge *g, double *out);

/* --------------------------------------------------------- vector algebra */

/*
 * out[i] = <v_i, w> = sum_k conj(v_i[k]) w[k] for i < nvec: the fused
 * multi-dot of the Gram-Schmidt step of FGMRES (Sec. 3.1).  v: nvec complex
 * FP64 vectors of n elements at stride ld elements; w: n elements;
 * out: nvec complex (device).  All device pointers; n <= 2^40, nvec <= 64.
 * Uses library-owned device scratch for the per-block partial sums.
 */
qdd_status qdd_cdot_multi(qdd_ctx *ctx, const double *v, int nvec, int64_t ld, const double *w, int64_t n,
                          double *out, void *stream);

/*
 * Allocation-free form of qdd_cdot_multi: the same multi-dot, computed by the
 * same kernels, for callers that must not allocate device memory -- for
 * example code whose device memory is all owned by its own pre-sized pool, or
 * a latency-critical loop that cannot afford the device-wide synchronisation
 * that cudaFree implies.  The paper has no counterpart; it is a service of
 * this library.  It needs no context and calls no cudaMalloc, cudaFree or
 * other allocating routine: its per-block partial sums live in one fixed
 * 128 KiB device array inside the library, present on every GPU that loads
 * the library until the process exits.  It runs on the current CUDA device.
 * The first call on a device looks up the array's address there (once per
 * device); make that first call before any stream capture.  Limits: nvec
 * 1..64, n 1..2^40, ld >= n; anything else returns QDD_EINVAL with a message.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  Nothing in
 * the array needs to start at zero; each call overwrites what it reads.
 * Arguments and layout as for qdd_cdot_multi.  Unlike the other entry points
 * this one does not wait for its result: it returns once its kernels are
 * queued on `stream`, and out is ready in that stream's order (synchronise the
 * stream, or order later work after it, before reading out).
 */
qdd_status qdd_cdot_multi_noalloc(const double *v, int nvec, int64_t ld, const double *w, int64_t n,
                                  double *out, void *stream);

/* ------------------------------------------------------------- host logic */

/* Average load of a colour half-sweep: x / ceil(x) with x = domains per
 * colour / slots (Sec. 3.5, "Inter-core parallelization"). */
double qdd_load_model(double n_domains_per_colour, double n_slots);

/* Working set of one domain in bytes (Sec. 3.3): per site 4 links (72 reals)
 * and 2 clover blocks (72 reals) stored with link_bytes bytes per real, plus
 * single-precision spinors: n_full on every site (24 reals) and n_even on
 * the even sites only (12 reals per site on average), times the domain
 * volume. */
double qdd_domain_working_set(const int dom[4], int link_bytes, int n_full, int n_even);

/*
 * The device layout of a lattice and domain shape (host logic only; no GPU
 * needed), for checking: site_of[i] (V entries) is the host site index of
 * internal index i = slot*Vd + s; nbl (Vd*8) the neighbour slot of each
 * domain site in direction k = 2*mu + (0 forward, 1 backward), wrapped into the
 * domain, with bit 15 set when the hop leaves the domain; nbd (Nd*8) the
 * neighbouring domain slot.  Any output may be NULL.  Domain slots are
 * colour-major (all domains of colour 0 first), sites parity-split.
 */
qdd_status qdd_layout(const int L[4], const int dom[4], int *site_of, uint16_t *nbl, int *nbd);

/* ------------------------------------------------------------------ tuning */

typedef struct {
    int dom[4];        /* fastest domain shape */
    int nmr;           /* its MR step count */
    int iters;         /* Arnoldi steps it needed */
    int n_tried;       /* candidates timed */
    double ms;         /* its time-to-solution (CUDA events) */
    double wave_load;  /* x/ceil(x), x = domains per colour / SMs (Sec. 3.5) */
} qdd_tune_result;

/*
 * Autotuner (the paper picks the domain size by cache capacity, Sec. 3.3, and
 * the MR step count by time-to-solution, Sec. 3.7): for every domain shape in
 * dom_candidates (n_dom x 4 ints), both Schwarz kernel variants where they
 * apply, and every MR step count in nmr_candidates (or p->nmr if n_nmr = 0),
 * build the gauge field, run the caller's solve (b: host layout, host or
 * device) once untimed and once timed, and return the fastest converged
 * setting.  log (may be NULL) receives a JSON array with every candidate's
 * time, iteration count and wave load.  Shapes the geometry rules reject are
 * logged and skipped.  Returns QDD_ENOCONV if no candidate converged.
 */
qdd_status qdd_autotune(qdd_ctx *ctx, const int L[4], const double *links, int links_on_device, double c_sw,
                        double kappa, const double *b, int b_on_device, const qdd_solve_params *p,
                        const int *dom_candidates, int n_dom, const int *nmr_candidates, int n_nmr,
                        qdd_tune_result *out, char *log, size_t log_len);

/* ---------------------------------------------------------------- serving */

/*
 * Asynchronous solve: enqueue (g, b, x, p) and return a ticket at once.  The
 * context's scheduler admits queued requests while the HBM budget and its
 * stream slots allow, runs admitted requests concurrently on separate
 * streams, and fills x (host layout, host memory that must stay valid until
 * the ticket completes).  b is copied at submit time.
 */
qdd_status qdd_submit(qdd_ctx *ctx, qdd_gauge *g, const double *b, double *x, const qdd_solve_params *p,
                      uint64_t *ticket);

/* Wait up to timeout_s seconds for a ticket.  QDD_OK / the solve's status
 * when done (rep filled, ticket retired); QDD_ENOTREADY if still running
 * after the wait; QDD_EINVAL for an unknown ticket. */
qdd_status qdd_poll(qdd_ctx *ctx, uint64_t ticket, qdd_report *rep, double timeout_s);

/* Serving-loop settings: max concurrently running requests (stream slots). */
qdd_status qdd_serve_config(qdd_ctx *ctx, int max_slots);

#ifdef __cplusplus
}
#endif

#endif /* QDD_H */
