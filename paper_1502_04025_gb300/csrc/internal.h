// Host-side internals of libqdd shared by its translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <complex>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/qdd.h"
#include "common.cuh"

namespace qdd {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
void clear_error();

#define QDD_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ::qdd::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return QDD_ECUDA;                                                                \
        }                                                                                    \
    } while (0)

#define QDD_TRY(expr)                   \
    do {                                \
        qdd_status s_ = (expr);         \
        if (s_ != QDD_OK) return s_;    \
    } while (0)

// ------------------------------------------------------------ kernel timing

enum KClass { K_SAP = 0, K_DSLASH = 1, K_BLAS = 2, K_OTHER = 3 };

// Launch bookkeeping of a context: launch counts always, CUDA-event timing of
// each launch when profiling is on (events resolved at sync points).
struct Timer {
    int mask = 0;  // classes timed with events
    long long launches[4] = {0, 0, 0, 0};
    double ms[4] = {0, 0, 0, 0};
    long long timed[4] = {0, 0, 0, 0};
    // algorithmic work of the launches (counted where a launcher states it)
    double flop[4] = {0, 0, 0, 0};
    double bytes[4] = {0, 0, 0, 0};
    struct Pending {
        cudaEvent_t a, b;
        int cls;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    std::mutex mu;

    cudaEvent_t get_event();
    void begin(int cls, cudaStream_t s, cudaEvent_t *a);
    void begin_seq(int cls, cudaStream_t s, cudaEvent_t *a);  // events, no launch count
    void count(int cls);                                      // launch count only
    void work(int cls, double f, double b);                   // add algorithmic flop and bytes
    void end(int cls, cudaStream_t s, cudaEvent_t a);
    void resolve();  // after the stream has been synchronised
    ~Timer();
};

struct LaunchScope {
    Timer &t;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    // timed = false: count the launch, but leave its timing to an enclosing
    // scope (a sequence of dependent launches timed as one, see SapScope)
    LaunchScope(Timer &t_, int cls_, cudaStream_t s_, bool timed = true) : t(t_), cls(cls_), s(s_)
    {
        if (timed) t.begin(cls, s, &a);
        else t.count(cls);
    }
    ~LaunchScope() { t.end(cls, s, a); }
};

// Events around a whole preconditioner application (2*ncy half-sweep launches
// that overlap through programmatic dependent launch); the time lands in the
// class without adding to its launch count.
struct SeqScope {
    Timer &t;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    SeqScope(Timer &t_, int cls_, cudaStream_t s_) : t(t_), cls(cls_), s(s_) { t.begin_seq(cls, s, &a); }
    ~SeqScope() { t.end(cls, s, a); }
};

// ------------------------------------------------------------------- memory

struct Ctx;

struct DevMem {
    Ctx *ctx = nullptr;
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    ~DevMem() { release(); }
    qdd_status alloc(Ctx *c, size_t n);
    qdd_status ensure(Ctx *c, size_t n) { return (bytes >= n && p) ? QDD_OK : alloc(c, n); }
    void release();
    template <typename T>
    T *as() const { return (T *)p; }
};

// ------------------------------------------------------------------ context

struct Request;

struct Ctx {
    int device = 0;
    int nsm = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    Timer timer;
    // scratch of the reductions (per-block partials), grown on demand
    DevMem red_scratch;
    std::mutex red_mu;
    // serving
    std::mutex q_mu;
    std::condition_variable q_cv, done_cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    std::vector<std::thread> workers;
    int max_slots = 4;
    int running = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    ~Ctx();
};

// ------------------------------------------------------------------ geometry

struct HostGeom {
    int L[4], dom[4], nb[4];
    int V, Vd, Vh, Nd, Nd2;
    std::vector<int> slot_block;   // slot -> block index
    std::vector<int> block_slot;   // lexicographic block index -> slot
    std::vector<int> site_of;      // internal index -> host site index
    std::vector<uint16_t> nbl;     // [Vd][8]
    std::vector<int> nbd;          // [Nd][8]
    std::vector<uint32_t> fcoord;  // [Vd]: byte mu = index of the site's coordinates transverse to mu
    int foff[8] = {0};             // first face slot of each direction
    int nf = 0;                    // face slots per domain
};

qdd_status make_geometry(const int L[4], const int dom[4], HostGeom &hg);

// A lower-precision copy of the fields the operator and the preconditioner read.
struct PrecCopy {
    bool valid = false;
    DevMem links, clov, clov_s, sclov, sclov_s;
    bool valid12 = false;
    DevMem links12;  // first two rows of each link, for the full-lattice operator
};

// Device and pinned host buffers of one solve (Krylov basis, preconditioner
// fields, scalars); reused across solves and grown on demand.
struct Workspace {
    int nrhs = 0, m = 0;
    qdd_prec sp = QDD_PREC_F32;
    DevMem io, b, x, V, Z, rho, rho_s, face, dev, scratch, err;
    DevMem ZR, Vt, ZRt, P;  // deflated restarts: recycled z (FP64), temporaries, P matrices
    double2 *host = nullptr;  // pinned mirror of `dev`
    size_t host_elems = 0;
    std::vector<double> hist;
    ~Workspace()
    {
        if (host) cudaFreeHost(host);
    }
};

// A gauge field sharded in t (qdd_create_gauge_field_slab): the rank's
// communication hooks, the extended lattice whose clover term the owned
// sites take, and the tables and buffers of the boundary exchanges.
struct Slab {
    qdd_comm comm{};
    int lt = 0, Ls = 0;        // local t extent, sites of one t plane
    qdd_gauge *ext = nullptr;  // (Lx, Ly, Lz, lt + 2 dom_t): one domain block of halo on each side
    DevMem ext_map;            // [V] internal index in ext of each owned site (clover remap)
    DevMem plane_base;         // [2][Ls] int64: internal element offset of component 0, planes 0 and lt-1
    DevMem last_link;          // [Ls] int64: element offset of U_t at plane lt-1 in the FP64 links
    DevMem bufs;               // [4][nrhs][Ls][6] double2: own backward push, own forward projection, received
    size_t buf_rhs = 0;
    // page-locked staging of the cyclic shifts: face slots, operator planes, sums
    void *host_face = nullptr, *host_op = nullptr, *host_red = nullptr;
    size_t face_bytes = 0, op_bytes = 0, red_bytes = 0;
    // the exchanges run on a side stream while the interior computes
    cudaStream_t side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool op_host_layout = false;  // the pending operator exchange's addressing
    ~Slab();
};

struct Gauge {
    Ctx *ctx = nullptr;
    std::unique_ptr<Slab> slab;  // set for a field sharded in t
    HostGeom hg;
    Geom geom{};
    DevMem d_nbl, d_nbd, d_site_of, d_block_slot, d_fcoord;
    DevMem links64;           // FP64 links, internal layout
    bool su3 = false;         // every link SU(3) to kSu3Tol
    bool two_rows = false;    // the FP32/16-bit full-lattice operator reads two rows per link
    bool have_clover = false;
    int sap_variant = 0;      // Schwarz kernel form (qdd_set_schwarz_variant)
    double csw = 0, kappa = 0;
    DevMem clov64, sclov64;   // FP64 clover A and Schwarz form (A even, A^-1 odd)
    PrecCopy copies[5];       // index = qdd_prec; F64 entry aliases the masters
    std::unique_ptr<Workspace> ws;  // workspace of the synchronous entry points
    std::unique_ptr<struct Staging> stage;  // buffers of apply_D / sap_apply, freed with the gauge
    std::shared_ptr<struct Multigrid> mg;  // two-level multigrid preconditioner (qdd_mg_setup)
    std::mutex mu;            // one synchronous call at a time per gauge object
    std::mutex copy_mu;       // guards the lazily built precision copies
    ~Gauge();
};

// Field pointers of a precision for the kernels.
template <typename S>
struct Fields {
    Field<S> U, A, C;  // links, clover, Schwarz clover
};

// Paired-plane order of a 16-bit field read only by the full-lattice
// operator: planes 2q and 2q+1 of a site are adjacent (one 8-byte load).
// Element index of plane p of site s in domain d, for P planes per site.
__host__ __device__ __forceinline__ int64_t pair_index(int64_t d, int P, int p, int Vd, int s)
{
    return (((int64_t)d * (P / 2) + p / 2) * Vd + s) * 2 + (p & 1);
}

qdd_status ensure_copy(Gauge *g, qdd_prec prec, cudaStream_t s);
// the two-row link copy of a storage precision (FP32, FP16, BF16)
qdd_status ensure_links12(Gauge *g, qdd_prec prec, cudaStream_t s);
// links whose unitarity and determinant deviate by more than this keep three rows
constexpr double kSu3Tol = 1e-10;

// storage of the spinors and of the links/clover copy a precision mode uses
inline qdd_prec spinor_store(qdd_prec p) { return p == QDD_PREC_H16 ? QDD_PREC_F32 : p; }
inline qdd_prec field_store(qdd_prec p) { return p == QDD_PREC_H16 ? QDD_PREC_F16S : p; }
inline bool is_sap_prec(qdd_prec p)
{
    return p == QDD_PREC_F64 || p == QDD_PREC_F32 || p == QDD_PREC_F16S || p == QDD_PREC_BF16S || p == QDD_PREC_H16;
}

// ------------------------------------------------------------- launchers

// layout.cu
qdd_status launch_links_to_internal(Gauge *g, const double *links_host_layout_dev, cudaStream_t s);
// host-layout FP64 spinors (device) <-> internal fields of storage prec
qdd_status launch_spinor_in(Gauge *g, const double *src, void *dst, float *dst_scale, qdd_prec prec, int nrhs,
                            cudaStream_t s);
qdd_status launch_spinor_out(Gauge *g, const void *src, const float *src_scale, double *dst, qdd_prec prec,
                             int nrhs, cudaStream_t s);
// internal -> internal precision conversion of spinors
qdd_status launch_spinor_convert(Gauge *g, const void *src, const float *src_scale, qdd_prec sp, void *dst,
                                 float *dst_scale, qdd_prec dp, int nrhs, cudaStream_t s);
// v = w / |w| (FP64, |w|^2 on the device) and its copy in a 16-bit storage
// (F16S / BF16S, per-site scale) in one pass, one right-hand side
qdd_status launch_scale_convert(Gauge *g, const double2 *w, const double2 *norm2, double2 *out64, void *dst,
                                float *dst_scale, qdd_prec dp, cudaStream_t s);
// plane-wise down-conversion of links (unscaled) / clover (per-site scale)
qdd_status launch_links_convert(Gauge *g, qdd_prec dp, void *dst, cudaStream_t s);
// paired: the full-lattice operator's copy (16-bit formats in paired-plane order)
qdd_status launch_clover_convert(Gauge *g, const double2 *src, qdd_prec dp, void *dst, float *dst_scale,
                                 cudaStream_t s, bool paired = false);
// *d_bad = 1 when some link is not SU(3) to tol; two-row copy of the links
qdd_status launch_su3_check(Gauge *g, double tol, int *d_bad, cudaStream_t s);
qdd_status launch_links12_convert(Gauge *g, qdd_prec dp, void *dst, cudaStream_t s);
// FP64 complex -> double-float (hi, lo) pairs
qdd_status launch_split_convert(Gauge *g, const double2 *src, float4 *dst, int64_t n, cudaStream_t s);

// clover.cu
qdd_status launch_clover_build(Gauge *g, double csw, double kappa, int *d_singular, cudaStream_t s);

// dslash.cu: out = D in (or out = b - D in when b != NULL); arith F64 or F32;
// in_prec/out_prec the storage of the spinors; link/clover storage = fields_prec.
qdd_status launch_dslash(Gauge *g, qdd_prec arith, qdd_prec fields_prec, const void *in, const float *in_s,
                         qdd_prec in_prec, void *out, float *out_s, qdd_prec out_prec, const double2 *b, int nrhs,
                         cudaStream_t s);

// sap.cu: one half-sweep over the domains of `colour`
struct SapBuffers {
    void *rho, *face, *psi;  // face: sap_face_bytes() of face slots
    float *rho_s;
};
// gather_only: apply the pending inter-domain update to the residual of the
// domains of `colour` and store it, without a block solve.
// pdl: launch as a programmatic dependent of the previous half-sweep (its
// CTAs may start early and stage read-only data; it must directly follow a
// half-sweep in the stream).  timed: bracket this launch with profiling
// events (false when the caller times a whole preconditioner application).
// Bytes of the face slots of all domains (the inter-domain update in flight).
size_t sap_face_bytes(const HostGeom &hg, qdd_prec prec, int nrhs);
// out-of-range indices skipped by the range-checked build's kernels (0 otherwise)
unsigned long long check_hits_sap();
qdd_status set_first_wait_spins_sap(unsigned spins);
unsigned long long check_hits_dslash();
unsigned long long check_hits_mg();
// part: 0 every domain of the colour; 1 those of the first and last t-block
// (a sharded field's boundary), 2 the others
qdd_status launch_sap_halfsweep(Gauge *g, qdd_prec prec, const SapBuffers &b, int colour, int nmr, int nrhs,
                                int first_psi, int gather, int gather_only, int *d_err, cudaStream_t s,
                                bool pdl = false, bool timed = true, int part = 0);
size_t sap_smem_bytes(const HostGeom &hg, qdd_prec prec, bool stage_links, bool stage_clover);

// blas.cu (FP64 complex vectors of n elements, stored as double2; scratch holds
// blas_scratch_elems(ctx) double2 of per-block partial sums)
int blas_blocks(const Ctx *ctx, int64_t n);
size_t blas_scratch_elems(const Ctx *ctx);
// allocates a reduction scratch buffer (if too small) with its block counter at zero
qdd_status blas_scratch_ensure(Ctx *ctx, DevMem &m);
qdd_status blas_cdot_multi(Ctx *ctx, const double2 *v, int nvec, int64_t ld, const double2 *w, int64_t n,
                           double2 *out, double2 *scratch, cudaStream_t s);
qdd_status blas_caxpy_multi_norm(Ctx *ctx, const double2 *v, int nvec, int64_t ld, const double2 *coef, double2 *w,
                                 int64_t n, double2 *norm2_out, double2 *scratch, cudaStream_t s);
qdd_status blas_norm2(Ctx *ctx, const double2 *w, int64_t n, double2 *out, double2 *scratch, cudaStream_t s);
// out = w / |w| from the squared norm on the device; out32 (optional) also gets
// the result rounded to FP32
qdd_status blas_scale_by_norm(Ctx *ctx, const double2 *w, int64_t n, const double2 *norm2, double2 *out,
                              cudaStream_t s, float2 *out32 = nullptr);
qdd_status blas_axpy_multi(Ctx *ctx, const void *z, bool z_f32, int nvec, int64_t ld, const double2 *coef,
                           double2 *x, int64_t n, cudaStream_t s);
// out_c (+)= sum_i src_i P[i*ldp + c], c < ncols (P on the device, row-major)
qdd_status blas_combine(Ctx *ctx, const void *src, bool src_f32, int nsrc, int64_t ld, const double2 *P, int ldp,
                        int ncols, double2 *out, int64_t ldo, int64_t n, int accumulate, cudaStream_t s);

// mg.cu: z = M_MG v, one right-hand side (v FP64, z in zp storage); the
// precision of the multigrid's Schwarz smoother
qdd_status mg_vcycle(Gauge *g, const double2 *v, void *z, qdd_prec zp, cudaStream_t s);
qdd_prec mg_smoother_prec(const Gauge *g);

// slab.cu: the exchanges of a field sharded in t (no-ops without a slab)
// sum n doubles of host memory over the ranks
qdd_status slab_allreduce(Gauge *g, double *host, size_t n);
// sum n complex values of device memory over the ranks (in place; synchronises s)
qdd_status slab_allreduce_dev(Gauge *g, double2 *dev, int n, cudaStream_t s);
// One Schwarz half-sweep of a sharded field, in the overlap order of Sec. 3.6:
// the domains of the first and last t-block first, then the interior, while
// the face slots the boundary domains pushed across the slab boundaries move
// to the neighbouring ranks on the side stream (when exchange is set); the
// next work on s waits for the received slots.
qdd_status slab_sap_halfsweep(Gauge *g, qdd_prec prec, const SapBuffers &b, int colour, int nmr, int nrhs,
                              int first_psi, int gather, int *d_err, cudaStream_t s, bool exchange);
// The operator on a sharded field: begin before the operator's launch (packs
// the boundary planes of in, FP64 or FP32, internal or host layout, on the
// side stream), end after it (the cyclic shift runs while the operator
// computes; then out, FP64 in the same layout, holding D in, or b - D in when
// residual, gets the neighbours' hops in place of the wrapped ones).
qdd_status slab_dslash_begin(Gauge *g, const void *in, bool in_f32, bool host_layout, int nrhs, cudaStream_t s);
qdd_status slab_dslash_end(Gauge *g, double2 *out, bool residual, int nrhs, cudaStream_t s);
// the clover of the owned sites from the extended lattice (after its build)
qdd_status slab_clover_remap(Gauge *g, cudaStream_t s);
qdd_status slab_setup(Gauge *g, qdd_gauge *ext, const qdd_comm &comm);
void slab_regions(const HostGeom &hg, int colour, int out[6]);

// solver.cu
std::unique_ptr<Workspace> make_workspace();
size_t workspace_bytes(const Gauge *g, int m, int nrhs, qdd_prec sp, bool use_sap, int kdr = 0);
size_t workspace_held(const Workspace *w);
void workspace_release(Workspace *w);
// every device allocation a solve with p makes: its workspace and the
// precision copies of the gauge field it reads (the serving loop makes them
// at admission, under its lock)
qdd_status solve_prepare(Gauge *g, Workspace *w, const qdd_solve_params *p, cudaStream_t s);
// rel_out (optional): true relative residual of every right-hand side at return
qdd_status solve_impl(Gauge *g, Workspace *w, const double *b, double *x, int on_device,
                      const qdd_solve_params *p, qdd_report *rep, cudaStream_t s,
                      std::vector<double> *rel_out = nullptr);

}  // namespace qdd

struct qdd_ctx : public qdd::Ctx {};
struct qdd_gauge : public qdd::Gauge {};
