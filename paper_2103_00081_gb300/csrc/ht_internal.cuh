// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ht.h"

namespace ht {

// ---------------------------------------------------------------------------
// Mesh description passed by value to every kernel.
// ---------------------------------------------------------------------------
struct Grid {
    int P;                      // element order (1 or 2)
    int ncx, ncy, ncz;          // cells per direction
    int Nx, Ny, Nz;             // nodes per direction (P*nc + 1)
    long long nn, nc;           // node and cell counts
    int dmask;                  // Dirichlet faces of the field (bit f = face f)
    // graded mesh: per-cell volume, 1/hx, 1/hy, 1/hz as [4][nc] (null: uniform)
    const double* geo64;
    const float* geo32;
};

// Reference-element constants for a uniform axis-aligned cell.
//   B[q][a], D[q][a]: 1D Lagrange values / derivatives (w.r.t. the reference
//   coordinate on [0,1]) at the (P+1) Gauss points.
//   W[q]: 3D Gauss weight times the cell volume.
//   G[d], Lam[d]: fast-diagonalisation factors of the 1D pair (k_d, m_d):
//   m_d = G^T G, k_d = G^T diag(Lam) G, so that the cell matrix
//   alpha M_e + beta K_e = (Gx (x) Gy (x) Gz)^T diag(alpha + beta*(Lx+Ly+Lz))
//   (Gx (x) Gy (x) Gz) -- sum factorisation in the 1D eigenbasis.
//   dM, dK: diagonals of the cell mass / stiffness matrices.
template <typename T>
struct Elem {
    T G[3][3][3];
    T Lam[3][3];
    T B[3][3];
    T D[3][3];
    T W[27];
    T invH[3];
    T dM[27];
    T dK[27];
    T LS[27];      // Lx[a] + Ly[b] + Lz[c] per mode l = a + n(b + n c)
    T dm1[3], dk1[3];   // diagonals of the 1D mass and stiffness of the unit cell (graded meshes)
};

// A float-float value hi + lo (|lo| <= ulp(hi)/2, about 48 significant bits),
// the arithmetic of the emulated-FP64 outer residuals (operators in ht_ops.cu).
struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df64(int v) : hi((float)v), lo(0.0f) {}
};

// Device-resident scalars of one Krylov solve.
struct Scal {
    double bb, rr, rz, rz_new, pq, alpha, beta;
    double rho, rho_old, omega, rv, ts, tt, rr0;
    double cheb_theta, cheb_delta;
    int done, iters, status, restarts;
    int kdone, conv;
    double rz2[2];   // r.z of the fused CG, indexed by iteration parity
    unsigned ticket; // CTAs done in the running fused-CG kernel (the last one resets it)
    double tol2;     // squared relative tolerance and iteration limit of the
    int max_iter;    // running solve (read by the fused kernels)
};

// GMRES(m) Hessenberg data (device resident).  H is column-major with
// leading dimension kMaxRestart + 1: H[j + (kMaxRestart + 1) * k].
constexpr int kMaxRestart = 512;
constexpr int kDotChunk = 32;     // basis vectors per CTA row in the multi-dot
struct Gmres {
    double H[(kMaxRestart + 1) * kMaxRestart];
    double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
    double hc[kMaxRestart + 1];   // second-pass corrections
    double inv;                   // 1 / norm of the newest basis vector
};

enum { ST_OK = 0, ST_BREAKDOWN = 1, ST_NAN = 2 };

}  // namespace ht

// zeros in front of the element buffers (E[-1] is the zero slot of node gathers)
constexpr int kElemPad = 64;

// profiling kinds: field (FP64 apply), field + 2 (FP32 apply), fused iterations
enum { HT_PROF_CG_ITER = 4, HT_PROF_BICGSTAB_ITER = 5, HT_PROF_KINDS = 6 };

// ---------------------------------------------------------------------------
// The context behind the opaque ht_ctx handle.
// ---------------------------------------------------------------------------
struct ht_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ht_mesh mesh{};
    ht::Grid grid{};
    double H[3] = {0, 0, 0};
    ht::Elem<double> e64{};
    ht::Elem<float> e32{};
    ht::Elem<ht::df64> edf{};               // e64 split into float pairs
    int num_sms = 0;

    // coefficients
    double* K64 = nullptr;
    float* K32 = nullptr;
    float* h32 = nullptr;                   // FP32 copy of h^{n+1} for the FP32 heat operator
    double* lam64 = nullptr;    // optional per-cell
    double* cT64 = nullptr;
    float* lam32 = nullptr;
    float* cT32 = nullptr;
    double lam_u = 0, cT_u = 0, cw = 0, Ss = 0;
    bool cells_set = false;

    // boundary conditions
    int bc_type[2][6] = {{0}};
    double bc_val[2][6] = {{0}};
    std::vector<double> bc_nodal[2][6];     // per-face-node values (empty: bc_val everywhere)
    int dmask[2] = {0, 0};
    double* g[2] = {nullptr, nullptr};     // nodal Dirichlet values (0 off the mask)
    bool bc_dirty = true;
    // Dirichlet faces whose value follows mean + amp sin(2 pi t / period + phase)
    struct Seasonal {
        int on = 0;
        double mean = 0, amp = 0, period = 1, phase = 0;
    };
    Seasonal seasonal[2][6];
    // pile surfaces held at a square-wave temperature (heat Dirichlet rows):
    // host rows [n][9] = x, y, z_top, z_bot, radius, T_mean, T_amp, period, phase
    std::vector<double> ptemp_rows;
    int n_ptemp_nodes = 0;                  // nodes held (the last pile listed wins a shared node)
    long long* ptemp_node = nullptr;
    int* ptemp_pile = nullptr;
    double* d_ptemp = nullptr;              // [n][4] T_mean, T_amp, period, phase
    // heat Dirichlet rows off the Dirichlet faces (pile surfaces), sorted
    int n_dint = 0;
    long long* dint = nullptr;
    std::vector<long long> dint_host;
    double* dint_a64 = nullptr;             // scratch of the wrapped operators
    double* dint_b64 = nullptr;
    float* dint_a32 = nullptr;

    // state
    double* h = nullptr;
    double* T = nullptr;
    double t = 0.0;

    // loads
    double* Fstat[2] = {nullptr, nullptr};   // time-independent nodal loads
    double* F[2] = {nullptr, nullptr};       // loads at the current step time
    double* extra[2] = {nullptr, nullptr};
    std::vector<ht_line_src> piles;
    std::vector<ht_box_src> boxes;
    std::vector<ht_well> wells;
    bool loads_dirty = true;
    int n_pile_nodes = 0;
    int* pile_node = nullptr;
    int* pile_off = nullptr;
    int* pile_src = nullptr;
    double* pile_w = nullptr;
    ht_line_src* d_piles = nullptr;
    int n_well_nodes = 0;
    int* well_node = nullptr;
    double* well_d = nullptr;               // c_w Q/L int N_i dz (heat, injection)
    double* wdn64 = nullptr;                // the same per node (0 elsewhere), for the fused solvers
    float* wdn32 = nullptr;

    // Darcy flux at Gauss points [3*nq^3][cells]
    double* qs64 = nullptr;
    float* qs32 = nullptr;
    // element-result buffers of the two-pass apply [(p+1)^3][cells]
    // graded mesh (tensor-product cell widths): face coordinates per axis
    // (empty: uniform cells of size H) and the per-cell geometry [4][nc]
    // (volume, 1/hx, 1/hy, 1/hz) on the device
    std::vector<double> faces[3];
    std::vector<double> widths[3];
    bool graded = false;
    bool geo_dirty = false;
    double* geo64 = nullptr;
    float* geo32 = nullptr;
    ht::df64* xdf = nullptr;                // float-float copies of the operand and the head for the
    ht::df64* hdf = nullptr;                // emulated-FP64 residuals (allocated on first use)
    double* E64 = nullptr;                  // element buffers: kElemPad zeros, then (P+1)^3 nc entries
    float* E32 = nullptr;

    // Krylov workspace
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double *b = nullptr, *D = nullptr, *rh = nullptr, *v = nullptr, *s = nullptr;
    double *tv = nullptr, *ph = nullptr, *sh = nullptr, *z2 = nullptr;
    float *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *D32 = nullptr, *rh32 = nullptr, *v32 = nullptr, *s32 = nullptr, *t32 = nullptr;
    float *ph32 = nullptr, *sh32 = nullptr, *zz32 = nullptr, *d32 = nullptr;
    double* part = nullptr;       // partial sums [8][part_stride]
    int part_stride = 0;
    ht::Scal* scal = nullptr;
    ht::Scal* scal_host = nullptr;  // pinned mirror
    ht::Gmres* gm = nullptr;        // [2]: FP64 solve, FP32 inner solve
    double* V64 = nullptr;          // GMRES basis (restart+1 vectors), lazily allocated
    float* V32 = nullptr;
    int V_m = 0;
    double cheb_lmax[2] = {0, 0};
    double cheb_dt[2] = {-1, -1};

    ht_solver_opts opts{};
    std::string err;

    // initial guesses extrapolated in time (HT_GUESS_EXTRAPOLATE): the fields
    // of the last completed steps, gpast[field][k] at time gtime[k] (k = 0 the
    // step before the current state), ghist of them valid (0..2)
    double* gpast[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double gtime[2] = {0.0, 0.0};
    int ghist = 0;
    bool guess_open = false;            // a batched step has rotated the head's past fields
    double guess_fast[2] = {-1.0, -1.0};   // FP32-operator residual of the guess in x (-1: unknown)

    // learned warm start
    ht_unet* net = nullptr;
    int learn_record = 0;
    int hist = 0;                       // increments stored (0..2)
    double *hn = nullptr, *Tn = nullptr;    // state at the start of the step
    double *dh1 = nullptr, *dh2 = nullptr, *dT1 = nullptr, *dT2 = nullptr;
    float *feat = nullptr, *targ = nullptr, *pred = nullptr;
    int Dp = 0, Hp = 0, Wp = 0;
    double lscale_T = 1.0, lscale_h = 1.0;   // RMS of the last increments (feature scales)
    int have_feat = 0, have_sample = 0;

    // launch accounting / apply timing
    long long n_launch = 0;
    int prof_on = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;                 // pairs in use
    std::vector<int> ev_kind;           // field + 2 * fp32 of each recorded pair
    std::vector<int> ev_weight;         // iterations covered by each recorded pair
    std::vector<std::vector<float>> prof_w = std::vector<std::vector<float>>(HT_PROF_KINDS);
    // CUDA graphs of kGraphIters fused Krylov iterations, recaptured when the
    // pointers or dt they were captured with change ([0] FP64, [1] FP32)
    struct FusedGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key[12] = {};
        double dt = 0.0;
        double ss = 0.0;                // operator scalars baked into the captured launches
    };
    FusedGraph g_cg[2], g_bi[2];
    FusedGraph g_cg1;                   // single-pass Q1 CG iteration (FP32)
    FusedGraph g_bi1;                   // single-pass Q1 BiCGStab iteration (FP32)
    // iterations of the inner solves of the last step, per field and outer
    // pass: the next solve checks convergence first near that count
    int iter_hint[2][8] = {};
    int cur_hint = 0;
    std::vector<std::vector<float>> prof_ms = std::vector<std::vector<float>>(HT_PROF_KINDS);
};

namespace ht {

// error helpers (host)
int fail(ht_ctx* c, int code, const char* fmt, ...);
#define HT_CUDA(ctx, call)                                                        \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess)                                                    \
            return ::ht::fail((ctx), HT_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, \
                              #call, cudaGetErrorString(e_));                     \
    } while (0)
#define HT_TRY(expr)              \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != HT_OK) return rc_; \
    } while (0)

constexpr int kVecBlocksPerSM = 4;
constexpr int kVecThreads = 256;
int vec_grid(const ht_ctx* c);

// ---- operator launchers (ht_ops.cu) ---------------------------------------
// Operator modes
enum { MODE_APPLY = 0, MODE_RHS = 1, MODE_DIAG = 2 };

// y = A0 x for the head (field 0) or heat (field 1) operator, FP64 or FP32.
// If dot_part != nullptr each tile writes sum_i x_i y_i into dot_part[tile].
// If sc != nullptr the kernels return at once when sc->done is set.
int launch_apply64(ht_ctx* c, int field, double dt, const double* x, double* y,
                   double* dot_part, int* n_part, const Scal* sc = nullptr);
int launch_apply32(ht_ctx* c, int field, float dt, const float* x, float* y,
                   double* dot_part, int* n_part, const Scal* sc = nullptr);
// b = lifted right-hand side of the next step of `field` (uses F[field]).
int launch_rhs(ht_ctx* c, int field, double dt, const double* u_old, double* b);
// D = diagonal of A0.
int launch_diag(ht_ctx* c, int field, double dt, double* D);
// the same in FP32 (the Jacobi scaling of the FP32 inner solves)
int launch_diag32(ht_ctx* c, int field, double dt, float* D);
// outer residual of the mixed form with the operator applied in float-float
// arithmetic: r32 = (float)(b - A x), partial sums of r.r and b.b in part
// (slots 0 and 1, *n_part entries); false if the two-pass buffers are absent
int launch_resid_df(ht_ctx* c, int field, double dt, const double* x, const double* b, float* r32,
                    double* part, int* n_part);
// r = b - q in FP64 with partial sums of r.r and b.b (slots 0, 1); reduction
// of those partial sums into c->scal[slot] (ht_krylov.cu)
int launch_resid64(ht_ctx* c, const double* b, const double* q, double* part, int* n_part);
int launch_norms(ht_ctx* c, int n_part, int slot);
// qs = -K grad h at Gauss points (both precisions).
int launch_darcy_qp(ht_ctx* c, const double* h);
// q at cell centres for output, component comp (0..2)
int launch_cell_flux(ht_ctx* c, const double* h, int comp, double* out);
// heat injection-well diagonal: y += dt * d .* x on the listed free nodes
int launch_well_apply64(ht_ctx* c, double dt, const double* x, double* y, const Scal* sc);
int launch_well_apply32(ht_ctx* c, float dt, const float* x, float* y, const Scal* sc);
int launch_well_diag(ht_ctx* c, double dt, double* D);
// F[field] = Fstat + extra + pile loads at time t
int launch_loads(ht_ctx* c, double t);
// Dirichlet values at time t of the seasonal faces and the pile surfaces
// (called by launch_loads with the step's t^{n+1}); ht_ops.cu
int launch_time_dirichlet(ht_ctx* c, double t);
// heat Dirichlet rows off the faces: the raw operator launches treat only
// the six faces; these wrap them (ht_ops.cu)
int dint_scatter(ht_ctx* c, double* dst, const double* src);   // dst[i] = src[i] on the rows
bool heat_fused_ok(const ht_ctx* c);    // no interior rows: the fused heat kernels apply
int apply_tiles(const ht_ctx* c);
// fused two-pass Jacobi-CG iteration of the head system (ht_ops.cu)
int fused_cg_iteration64(ht_ctx* c, double dt, double* x, double* r, const double* Dinv, double* p, Scal* sc,
                         int first);
int fused_cg_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* Dinv, float* p, Scal* sc,
                         int first);
bool fused_cg_available(const ht_ctx* c, int fp32);
// single-pass Jacobi-CG iteration of the Q1 head system in FP32 (ht_q1.cu):
// reads r, p (halos included) and writes r_out, p_out (the next iteration
// swaps them); x is updated in place.  first = 1 only forms the scalars of
// the start (x unchanged, r_out = r, p_out = D^-1 r)
bool q1_cg_available(const ht_ctx* c, int fp32);
int q1_cg_iteration32(ht_ctx* c, float dt, float* x, const float* r, const float* p, float* r_out, float* p_out,
                      Scal* sc, int first);
// Persistent single-pass CG of the inner FP32 head solves of many Q1
// problems (ht_q1.cu; used by the batched step).  prepare builds the work
// list of (problem, tile, z chunk) items and the per-problem descriptors for
// step size dt; planes > 0 fixes the node planes per z chunk (0: chosen from
// the batch's total work and the co-resident CTAs).  run makes one
// cooperative launch that performs the first pass and up to max_iter
// iterations of every problem whose inner scalars (slot 1) are not done,
// with grid-barrier waits bounded by budget clock cycles; *running receives
// the problems still running at the end and *err_cta the CTA whose wait ran
// out (-1 when none did; then the call returns HT_ETIMEOUT).  drop_cta >= 0
// makes that CTA leave at its first barrier without arriving (a failure
// injection for tests).
struct Q1Batch {
    void* d_probs = nullptr;
    int* d_items = nullptr;
    void* d_sync = nullptr;
    void* h_sync = nullptr;
    int nprob = 0, nitems = 0, grid = 0, planes = 0;
    int cap_probs = 0, cap_items = 0;
    double dt = -1.0;
};
int q1_batch_prepare(Q1Batch& q, ht_ctx* const* probs, int n, double dt, int planes, cudaStream_t st,
                     std::string* err);
int q1_batch_run(Q1Batch& q, cudaStream_t st, int max_iter, long long budget, int drop_cta, int* running,
                 int* err_cta, std::string* err);
void q1_batch_free(Q1Batch& q);
// single-pass heat applies of the Q1 BiCGStab iteration in FP32 (ht_q1.cu):
// reads p_in, v_in (halos included), writes p_out, v_out, t; then x, r
bool q1_bicgstab_available(const ht_ctx* c);
int q1_bicgstab_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* rh, const float* p_in,
                            const float* v_in, float* p_out, float* v_out, float* t, const float* Dinv, Scal* sc);
// pointwise BiCGStab update of x and r with the next beta (ht_ops.cu)
int launch_fbi_update32(ht_ctx* c, float* x, float* r, const float* p, const float* v, const float* t,
                        const float* Dinv, const float* rh, Scal* sc);
// fused two-pass Jacobi-BiCGStab iteration of the heat system (ht_ops.cu)
int fused_bicgstab_iteration64(ht_ctx* c, double dt, double* x, double* r, const double* rh, double* p, double* v,
                               double* t, const double* Dinv, Scal* sc);
int fused_bicgstab_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* rh, float* p, float* v,
                               float* t, const float* Dinv, Scal* sc);
// event bracketing of apply launches (kind = field + 2 * fp32)
int prof_begin(ht_ctx* c, int kind);
int prof_end(ht_ctx* c);
int prof_end_weighted(ht_ctx* c, int weight);   // the pair covers `weight` iterations
void prof_drop_last(ht_ctx* c);                 // forget the last pair (not yet flushed)
int prof_flush(ht_ctx* c);

// ---- allocation-free head apply (ht_ops.cu) ----------------------------------
constexpr int kNoAllocMaxTiles = 4096;     // partial sums held by the static scratch
constexpr int kNoAllocMaxDevices = 64;
int noalloc_head_apply_dot(const Grid& g, const Elem<double>& e, double Ss, double dt, const double* K,
                           const double* x, double* y, double* xAx, int device, cudaStream_t stream, char* msg,
                           size_t msg_len);

// ---- learned warm start (ht_learned.cu) --------------------------------------
constexpr int kLearnFeatures = 8;   // input channels of the network (see ht_learned.cu)
int learned_begin(ht_ctx* c);                                   // features + prediction
int learned_gate(ht_ctx* c, int field, double dt, double* x, const double* b, int* used, double* res);
int learned_end(ht_ctx* c);                                     // targets + history
void learned_free(ht_ctx* c);

// ---- Krylov (ht_krylov.cu) -------------------------------------------------
int solve_head(ht_ctx* c, double dt, double* x, const double* b, int* iters, int* outer, double* res);
int solve_heat(ht_ctx* c, double dt, double* x, const double* b, int* iters, int* outer, double* res);
int true_residual(ht_ctx* c, int field, double dt, const double* x, const double* b, double* rel);
// ||b - A x|| / ||b|| with A applied by the FP32 operator (FP64 right-hand side,
// exact Dirichlet rows): a cheap ranking of initial guesses
int fast_residual(ht_ctx* c, int field, double dt, const double* x, const double* b, double* rel);
int set_dirichlet_values(ht_ctx* c, int field, double* x);
// the extrapolated initial guess of a step to t1 (HT_GUESS_EXTRAPOLATE): when
// past fields are kept, forms their Lagrange extrapolation with the current
// field into z (Dirichlet values set) and reports its degree in *deg (0: none
// formed); in any case records the current field as the newest past one.
// The caller commits the new history with guess_commit after the step.
int guess_extrapolate(ht_ctx* c, int field, double t1, double* z, int* deg);
void guess_commit(ht_ctx* c, double t_prev);
void guess_free(ht_ctx* c);

}  // namespace ht
