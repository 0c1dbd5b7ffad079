// Internal declarations of libhyel: context, device layouts, kernel launchers.
//
// Device layouts (all owned by the context):
//   * Element data, structure-of-arrays over elements e (coalesced per thread):
//     geo[k*E + e] for k = 0..11 the reference shape-function gradients
//     g[A][I] = dN_A/dX_I, k = 12 the volume V, k = 13 tau_M.
//   * Block pattern "SELL-32": rows (nodes) grouped in slices of 32; slice s
//     owns slice_len[s] block columns starting at slice_ptr[s]; the block in
//     slice column b for row lane t (row = 32 s + t) lives at slot b*32 + t.
//     Column indices col[slot] (int32); a row's valid entries come first
//     (ascending column), padding repeats the row's own index with zero values.
//   * Block values in component-major order per 32-slot group, so that a warp
//     reading one component of 32 consecutive rows issues one coalesced load:
//     A[(b*9 + r*3 + c)*32 + t], B[(b*3 + r)*32 + t], C[(b*3 + c)*32 + t],
//     D[b*32 + t].
//   * Assembly staging: per element 18 records of 16 doubles (128 B each):
//     records 0..15 are the node pairs (a,b) -> [A 9 | B 3 | C 3 | D 1],
//     record 16 the element residual [a][R_m x,y,z | R_p], record 17 the
//     K_{.,udot} R_k correction in the same form. Record (e, k) sits at
//     stage[(((e >> 5) * 18 + k) * 32 + (e & 31)) * 16].
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "hyel.h"

namespace hyel {

constexpr int kRecords = 18;
constexpr int kRecordDoubles = 16;

// Throws are confined to host code; every C-ABI entry point converts them to
// a status code and a message.
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define HYEL_CK(call) ::hyel::check_cuda((call), #call)

// Device error word bits (set by kernels, read by the host at sync points).
enum : unsigned { ERR_INVERTED = 1u, ERR_NAN = 2u, ERR_SINGULAR = 4u };

// Grid-barrier words of the persistent (cooperative) kernels, one 128-byte
// line each: arrivals, release, abort (cleared before every launch) and the
// control line (wait limit in ns as a 64-bit word at kBarCtl, an injected
// fault at kBarCtl + 2, the address of the context's control line as a 64-bit
// word at kBarCtl + 4), copied from the context before every launch.
constexpr int kBarArrive = 0, kBarRelease = 32, kBarAbort = 64, kBarWords = 96;
constexpr int kBarCtl = 96, kBarAlloc = 128;

struct DeviceMesh {
    int64_t N = 0, E = 0, nnzb = 0;
    int32_t nslices = 0;
    int64_t ncols = 0;   // total slice columns
    int64_t nslots = 0;  // ncols * 32
    int32_t n_fibres = 0;
    int32_t vol_model = 0;
    double rho0 = 0, kd = 0, body[3] = {0, 0, 0};
    // traction and Dirichlet ramp
    double t_ramp = 1.0;
    // device arrays
    int4 *tets = nullptr;        // [E]
    double *geo = nullptr;       // [14][E]
    double *mat = nullptr;       // [4][E]: mu, kappa, k1, k2
    double *fib = nullptr;       // [6][E]: a1, a2 (n_fibres == 2)
    int32_t *slice_ptr = nullptr;  // [nslices + 1]
    int32_t *col_slice = nullptr;  // [ncols]: slice owning each slice column
    int32_t *row_len = nullptr;    // [N]
    int32_t *col = nullptr;        // [nslots]
    int32_t *diag_slot = nullptr;  // [N]
    int32_t *mirror = nullptr;     // [nslots]: slot of (c, r) for slot (r, c); -1 on padding
    int32_t *slot_ptr = nullptr;   // [nslots + 1]
    int32_t *slot_list = nullptr;  // [16 E]: staging record index e*18 + pair
    int32_t *node_ptr = nullptr;   // [N + 1]
    int32_t *node_list = nullptr;  // [4 E]: e*4 + a
    uint8_t *dir = nullptr;        // [N] bit c set if component c is constrained
    double *dir_val = nullptr;     // [3N] prescribed value at full ramp
    double *trac = nullptr;        // [3N] int N_A H dGamma at full load
    // host copies for downloads
    std::vector<int32_t> h_row_ptr, h_col;  // block CSR
    std::vector<int64_t> h_csr_slot;        // CSR position -> slot
    std::vector<double> h_hmax;             // longest reference edge per element (tau_M updates)
    std::vector<double> h_X;                // [3N] reference coordinates (multigrid rigid-body modes)
    double c_m = 1e-3;
};

struct DeviceMatrix {
    double *A = nullptr, *B = nullptr, *C = nullptr, *D = nullptr;      // assembled
    double *As = nullptr, *Bs = nullptr, *Cs = nullptr, *Ds = nullptr;  // scaled FP64
    float *Af = nullptr, *Bf = nullptr, *Cf = nullptr, *Df = nullptr;   // scaled FP32
    // scaled A as BF16 x per-block FP32 scale, one record per slot q:
    // Ah8[q] = entries 0..7 (row-major, two per 32-bit word), Ah1[q] = entry 8,
    // Ahs[q] = scale s = max |entry| (0 for padding)
    uint4 *Ah8 = nullptr;
    uint16_t *Ah1 = nullptr;
    float *Ahs = nullptr;
    // right-preconditioned operator of the A-solves, A~ = A M^-1 with M the
    // 3x3 block diagonal of the scaled A: FP64, FP32 and BF16-with-scale copies
    // in the layouts of As, Af and Ah8/Ah1/Ahs
    double *Ams = nullptr;
    float *Amf = nullptr;
    uint4 *Amh8 = nullptr;
    uint16_t *Amh1 = nullptr;
    float *Amhs = nullptr;
    double *w = nullptr;        // [4N] scaling
    double *jac64 = nullptr;    // [9][N] inverses of scaled diagonal blocks of A
    double *rdiag64 = nullptr;  // [3N] 1 / (scalar diagonal of the scaled A)
    float *jac32 = nullptr;
    double *shat64 = nullptr;   // [N] 1 / diag(S^) of the scaled system
    float *shat32 = nullptr;
    // symmetrized scaled A, A_sym = (A + A^T)/2, in the layout of As, and the
    // inverses of its 3x3 diagonal blocks (the CG inner solve), built on demand
    double *Asym64 = nullptr;
    float *Asym32 = nullptr;
    double *jsym64 = nullptr;   // [9][N]
    float *jsym32 = nullptr;
    // transposed operator [[A^T, C^T], [B^T, D^T]] in the same pattern: block
    // (i, c) holds A(c, i)^T, C(c, i), B(c, i), D(c, i)
    double *At = nullptr, *Bt = nullptr, *Ct = nullptr, *Dt = nullptr;
    bool assembled = false;
    bool scaled = false;
    bool amg_ready = false;   // multigrid operators built from the current scaled A
    bool shat_ready = false;    // explicit S^ (FP32) and its interval built from the current scaled blocks
    bool shat64_ready = false;  // ... and its FP64 copy
    bool asym_ready = false;    // A_sym and its block-Jacobi inverses built from the current scaled A
    bool acheb_ready = false;   // the A-Chebyshev interval of the current scaled A
    bool transposed = false;  // At..Dt hold the transpose of the current assembly
};

struct GmState {
    int done;       // stop iterating in this cycle
    int converged;  // res <= tol
    int k;          // iterations completed in the current cycle
    int flags;      // 1 = NaN/Inf, 2 = breakdown
    double beta, bnorm, tol, res, inv_scale;
};

struct Profile {
    bool on = false;
    struct Rec {
        cudaEvent_t a, b;
        int cls;
        double bytes;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double ms[HYEL_K_NCLASSES] = {0};
    int64_t launches[HYEL_K_NCLASSES] = {0};
    double bytes[HYEL_K_NCLASSES] = {0};
};

// Chebyshev interval of M^-1 A (HYEL_APREC_CHEB) and the FP32 scratch of its
// Arnoldi run and of the stand-alone apply (solver.cu)
struct AChebState {
    double *bounds = nullptr;   // device [2]: lmin, lmax
    double h_bounds[2] = {0.0, 0.0};
    float *V = nullptr;         // [(steps + 1) 3N]
    float *U = nullptr;         // [3 x 3N]: two directions and M w
    double *H = nullptr;        // [(steps + 1) steps]
    double *partial = nullptr;  // [2][steps + 1][grid]
    unsigned *bar = nullptr;
    double *work = nullptr;     // [3N] residual of the stand-alone apply
    float *dwork = nullptr;     // [2 x 3N] its directions
};

struct Workspace;  // Krylov workspaces (solver.cu)
struct Amg;        // multigrid hierarchy of the A-solves (amg.cu)

// Explicit S^ = D - C diag(A)^-1 B of the scaled system (§4.2) on the
// distance-2 node pattern, SELL-32 like the block pattern: entry p of row i at
// slot (slice_ptr[i / 32] + p) * 32 + i % 32, columns ascending, padding with
// column i and value 0 (schur_hat.cu).
struct SchurHat {
    int64_t nnz = 0, ncols = 0, nslots = 0, ncontrib = 0;
    int32_t max_row = 0;
    int32_t *slice_ptr = nullptr;  // [nslices + 1]
    int32_t *row_len = nullptr;    // [N]
    int32_t *col = nullptr;        // [nslots]
    // contributions of row i, in the order the numeric kernel visits them
    // (for each block slot (i, k): D_ik, then C_ik A_kk^-1 B_kj for each
    // block slot (k, j)): cptr[i] .. cptr[i + 1] - 1, pos = entry index in row i
    int64_t *cptr = nullptr;       // [N + 1]
    uint16_t *pos = nullptr;       // [ncontrib]
    double *v64 = nullptr;         // [nslots] (summed on demand)
    float *v32 = nullptr;          // [nslots] (the solver's copy)
    // Chebyshev interval from the Ritz values of diag(S^)^-1 S^: lmin, lmax
    double *bounds = nullptr;      // device [2]
    double h_bounds[2] = {0.0, 0.0};
    // scratch of the Arnoldi run (FP32) and the stand-alone Chebyshev apply
    double *work = nullptr;        // [3N] (Arnoldi: two FP32 directions and |diag(S^)|^-1/2)
    float *arn_V = nullptr;        // [(steps + 1) N]
    double *arn_H = nullptr;       // [(steps + 1) steps]
    double *partial = nullptr;     // [2][steps + 1][grid]
    unsigned *bar = nullptr;       // barrier words
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    DeviceMesh mesh;
    DeviceMatrix mat;
    double *stage = nullptr;     // staging records
    double *vec = nullptr;       // scratch nodal vectors (see newton.cu)
    double *red = nullptr;       // reduction partials
    unsigned *counter = nullptr; // last-block counters
    unsigned *err = nullptr;     // device error word
    unsigned *h_err = nullptr;   // pinned mirror
    double *h_red = nullptr;     // pinned scalars
    Workspace *ws = nullptr;
    Amg *amg = nullptr;
    SchurHat *sh = nullptr;
    AChebState *ach = nullptr;
    // set by the Newton step after its first correction: the Chebyshev
    // intervals (S^ and A) estimated at the first iteration are kept
    bool keep_intervals = false;
    Profile prof;
    size_t bytes_held = 0;
    int num_sms = 152;
    std::vector<void *> allocations;
    // control line of the grid barriers (see kBarCtl): device [32] words,
    // owned apart from `allocations` (it outlives mesh replacements)
    unsigned *ctl = nullptr;
};

// Clears the barrier words of one persistent launch and copies the context's
// control line (wait limit, injected fault) beside them, in stream order.
void bar_reset(Ctx &c, unsigned *bar);

// process-wide count of kernel launches issued by this library; while a graph
// is being recorded (g_capture_count set) launches are counted there instead
void count_launch();
extern thread_local int *g_capture_count;

// memory helpers
void *dalloc(Ctx &c, size_t bytes);
void dfree_all(Ctx &c);
template <typename T>
T *dalloc_n(Ctx &c, size_t n) { return static_cast<T *>(dalloc(c, n * sizeof(T))); }

// profiling
void prof_begin(Ctx &c, int cls, cudaEvent_t *ev);
void prof_end(Ctx &c, int cls, cudaEvent_t ev, double bytes);

// mesh.cu
void mesh_upload(Ctx &c, int64_t N, const double *X, int64_t E, const int32_t *tets,
                 const hyel_bc *bc, const hyel_material *mat);

// assemble.cu
struct TimeConsts {
    double am, af, gam, dt, c1, c2;  // c1 = af*gam*dt, c2 = c1^2/am
    double t_alpha, load;            // load factor s(t_alpha)
    int literal;
    int skip_corr = 0;  // R_k is zero up to rounding (after a corrector update): no K_{.,udot} R_k term
};
TimeConsts time_consts(const DeviceMesh &m, const hyel_time_params &tp);
// Assembles residual, rhs, tangent; returns the norms (host) when norms != nullptr.
// tangent = false: residual and norms only (no rhs, the matrix is left as it was).
void assemble(Ctx &c, const TimeConsts &tc, const hyel_state &st, double *res_out, double *rhs_out,
              double *norms4, bool tangent = true);
void matrix_download(Ctx &c, int32_t *row_ptr, int32_t *col, double *A, double *B, double *C, double *D);

// amg.cu
void amg_free(Ctx &c);
void amg_numeric(Ctx &c);  // builds the hierarchy on first use, then the level operators
int amg_levels(const Ctx &c, int64_t *sizes, int max);  // per level: block-nodes, stored blocks; returns levels
template <typename T>
void amg_apply(Ctx &c, const T *v, T *z);  // z = V-cycle(v), [3N]

// schur_hat.cu
void shat_free(Ctx &c);
template <typename V>
void shat_numeric(Ctx &c);  // builds the pattern on first use, then the V values of the current scaled blocks
void shat_ensure64(Ctx &c);  // the FP64 values, if not yet summed for this assembly
template <typename T>
void shat_spmv(Ctx &c, const T *x, T *y);  // y = S^ x, [N]

// sparse.cu
void solve_setup(Ctx &c);
void transpose_assembled(Ctx &c);  // fills At..Dt from A..D (mirror slots)
void asym_setup(Ctx &c);  // A_sym = (As + As^T)/2 and its diagonal-block inverses, unless current
// SpMVs. The *_ind forms take kd = (k, done) of a Krylov level (the first two
// ints of its device state): they write basis column k+1 (column stride given)
// and do nothing once the level is done; kd == nullptr means plain pointers.
template <typename T>
void spmv_A(Ctx &c, const T *Av, const T *x, T *y);
template <typename T>
void spmv_A_ind(Ctx &c, const T *Av, const T *x, T *y, int64_t ystride, const int *kd);
// A-SpMV on a BF16-with-block-scale copy (see HYEL_PREC_BF16S)
void spmv_A16_ind(Ctx &c, const uint4 *h8, const uint16_t *h1, const float *hs, const float *x, float *y,
                  int64_t ystride, const int *kd);
void spmv_full64(Ctx &c, const double *A, const double *B, const double *C, const double *D, const double *x,
                 double *y);
void spmv_full64_ind(Ctx &c, const double *A, const double *B, const double *C, const double *D, const double *x,
                     double *y, int64_t stride, const int *kd);  // x column k -> y column k+1
template <typename T>
void spmv_B(Ctx &c, const T *B, const T *xp, T *yv, const T *r);   // yv = r - B xp (r null: yv = B xp)
template <typename T>
void spmv_C(Ctx &c, const T *C, const T *xv, T *yp, const T *r);   // yp = r - C xv (r null: C xv)
template <typename T>
void spmv_D(Ctx &c, const T *D, const T *xp, T *yp);
template <typename T>
void spmv_DC_ind(Ctx &c, const T *D, const T *C, const T *xp, const T *xv, T *yp, int64_t ystride,
                 const int *kd);  // D xp - C xv

// solver.cu
void solve_nested(Ctx &c, const hyel_solver_params &p, const double *rhs, double *x, hyel_solve_stats *st);
void schur_apply(Ctx &c, const hyel_solver_params &p, const double *x, double *y, hyel_solve_stats *st);
void block_precond_apply(Ctx &c, const hyel_solver_params &p, const double *r, double *z, hyel_solve_stats *st);
void free_workspace(Ctx &c);
void shat_bounds(Ctx &c);  // Chebyshev interval of diag(S^)^-1 S^ from Arnoldi Ritz values (host-checked)
void shat_setup(Ctx &c);  // solve_setup, then S^ and its bound unless current
void shat_cheb_apply(Ctx &c, int matrix, int degree, double ratio, const double *x, double *y);
void acheb_setup(Ctx &c);  // solve_setup, then the A-Chebyshev interval unless current
void acheb_apply(Ctx &c, int degree, const double *x, double *y);
void acheb_free(Ctx &c);

// adjoint.cu
void solve_nested_transpose(Ctx &c, const hyel_solver_params &p, const double *rhs, double *x,
                            hyel_solve_stats *st);
void spmv_transpose(Ctx &c, const double *x, double *y);
void param_sensitivity(Ctx &c, const hyel_state &st, const double *lam, double *grad);
void adjoint_step(Ctx &c, const hyel_time_params &tp, const hyel_solver_params &sp, const hyel_state &sn,
                  const hyel_state &s1, double *ybar, double *ydbar, double *grad, double *lam_out,
                  hyel_solve_stats *stats);
void update_material(Ctx &c, const hyel_material *mat);

// probe.cu: launches the FP64 FMA probe; returns the flops of the launch
double fp64_fma_probe(Ctx &c, int64_t iters, double *sink);
void stream_read_probe(Ctx &c, const void *buf, int64_t bytes, double *sink);

// noalloc.cu
void residual_norm_static(Ctx &c, int matrix, const double *x, const double *b, double *out);

// newton.cu
void newton_step(Ctx &c, const hyel_time_params &tp, const hyel_solver_params &sp, hyel_state &s,
                 hyel_newton_stats *st);

// launch geometry
inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace hyel
