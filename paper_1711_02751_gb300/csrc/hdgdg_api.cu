// C ABI and host driver of the IMEX HDG-DG hot path (Algorithm 1 of arXiv:1711.02751).
//
// Host side: GLL tables, mesh geometry and the bottom are prepared on the CPU once; every
// per-stage operation runs in the CUDA kernels of this library.  One time step of
// Algorithm 1:
//   for each stage i: if a~_ii = 0 then Q = q^n
//                     else R1 = q^n + sum_{j<i} (a_ij dtM^{-1}NL_j + a~_ij dtM^{-1}L_j)  (combine)
//                          g = -C A^{-1} R1                                          (condense)
//                          S qhat = g by block-Jacobi GMRES(m)                          (Krylov)
//                          Q = A^{-1}(R1 - B qhat), dtM^{-1}L_i = (Q - R1)/a~_ii        (recover)
//                     dtM^{-1}NL_i = dt M^{-1} NL(Q)                                    (DG residual)
//   q^{n+1} = q^n + sum_i (b_i dtM^{-1}NL_i + b~_i dtM^{-1}L_i)                          (combine)
// The identity M^{-1} L_i = (Q - R1)/(dt a~_ii) holds exactly for the recovered Q because
// the local rows of the stage system are solved exactly (eq. IMEXRKDiscretizedForm).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <utility>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hdgdg.h"
#include "internal.h"

using namespace hdgdg;

namespace {

constexpr int kMaxStages = 5;

struct Plan {
    size_t n = 0, nt = 0;
    int NV = 0, NF = 0, NT = 0, m = 0, s = 0;
    size_t persistent = 0, setup_temp = 0;
};

constexpr int kMaxRestart = 31;   // the fused Gram-Schmidt kernels keep up to 32 basis vectors in registers

bool valid(const hdgdg_config* c) {
    return c && c->n_side >= (c->boundary != HDGDG_PERIODIC ? 1 : 2) && c->n_side <= 32768 && c->degree_k >= 1 && c->degree_k <= kMaxP - 1 &&
           std::isfinite(c->g) && c->g > 0.0 && std::isfinite(c->H0) && std::isfinite(c->dt) &&
           c->dt > 0.0 && c->scheme >= HDGDG_ARS2 && c->scheme <= HDGDG_RK3 &&
           (c->precision == HDGDG_FP64 || c->precision == HDGDG_MIXED) &&
           (c->linear_only == 0 || c->linear_only == 1) &&
           c->boundary >= HDGDG_PERIODIC && c->boundary <= HDGDG_VORTEX && std::isfinite(c->x0) &&
           std::isfinite(c->length) && c->batch >= 0 && c->batch <= (1 << 20) &&
           c->krylov_restart <= kMaxRestart && c->local_precision >= HDGDG_LOCAL_FP64 &&
           c->local_precision <= HDGDG_LOCAL_BF16_SPLIT &&
           ((c->local_precision != HDGDG_LOCAL_BF16 && c->local_precision != HDGDG_LOCAL_BF16_SPLIT) ||
            c->degree_k <= 4) &&   // tensor-core tiles: k <= 4
           c->krylov_guess >= -1 && c->krylov_guess <= 6 && (c->spmv_kernel == 0 || c->spmv_kernel == 1) &&
           (c->krylov_ortho == 0 || c->krylov_ortho == 1) && (c->residual_f32x2 == 0 || c->residual_f32x2 == 1) &&
           (c->local_dense == 0 || c->local_dense == 1) && (c->trace_operator == 0 || c->trace_operator == 1) &&
           (c->host_steps == 0 || c->host_steps == 1) &&
           (c->krylov_guess_ls == 0 || (c->krylov_guess_ls == 1 && c->precision == HDGDG_MIXED && c->krylov_guess >= 0)) &&
           (c->dg_precision == 0 || (c->dg_precision == 1 && c->precision == HDGDG_MIXED && c->degree_k <= 4)) &&
           (c->trace_operator == 0 ||
            (c->precision == HDGDG_MIXED && c->local_precision == HDGDG_LOCAL_F32X2 && !c->local_dense &&
             c->scheme != HDGDG_RK2 && c->scheme != HDGDG_RK3));
}

// the mixed form's trace solve applies S M^{-1} element by element (kernels_mf.cu)
bool matrix_free(const hdgdg_config* c) { return c->trace_operator == 1; }

bool explicit_scheme(const hdgdg_config* c) { return c->scheme == HDGDG_RK2 || c->scheme == HDGDG_RK3; }

int restart_of(const hdgdg_config* c) { return c->krylov_restart > 0 ? c->krylov_restart : 10; }

// order of the trace-solve initial guess (0: start from zero)
int guess_order(const hdgdg_config* c) { return c->krylov_guess < 0 ? 0 : c->krylov_guess == 0 ? 5 : c->krylov_guess; }

// local solves through the Schur complement on phi (FP64 and FP32-pair local arithmetic)
bool local_schur(const hdgdg_config* c) {
    return !c->local_dense && (c->local_precision == HDGDG_LOCAL_FP64 || c->local_precision == HDGDG_LOCAL_F32X2);
}

Plan make_plan(const hdgdg_config* c) {
    Plan p;
    const size_t N = (size_t)c->n_side, P = (size_t)c->degree_k + 1;
    const size_t B = c->batch > 0 ? (size_t)c->batch : 1;
    const size_t n_el = B * N * N, Np = P * P;
    const size_t n_edges = B * (c->boundary != HDGDG_PERIODIC ? 2 * N * (N + 1) : 2 * N * N);
    p.n = n_el * Np;
    p.NV = (int)(3 * Np);
    p.NF = (int)(3 * P);
    p.NT = (int)(12 * P);
    p.nt = n_edges * p.NF;
    p.m = restart_of(c);
    p.s = c->scheme == HDGDG_ARS2 ? 3 : c->scheme == HDGDG_ARS3 ? 5 : 3;
    const size_t d = sizeof(double);
    size_t b = 0;
    if (explicit_scheme(c)) {   // state, three stage increments, two stage states, face fluxes
        b += p.n * d + n_edges * P * d;
        b += 7 * 3 * p.n * d + p.nt * d;
        b += (reduction_scratch_doubles(p.m, (int)n_edges, (int)P) + mass_scratch_doubles() + 4 * (size_t)(p.m + 2) + 16) * d + 64;
        p.persistent = b;
        p.setup_temp = 0;
        return p;
    }
    b += p.n * d + n_edges * P * d + B * d;                   // phiB, tau, time-step factors
    b += n_el * (size_t)p.NV * p.NV * d;                      // A^{-1}
    b += n_edges * 6 * (size_t)p.NF * p.NF * d;               // S~
    b += n_edges * 6 * sizeof(int);                           // columns
    b += 2 * n_edges * (size_t)p.NF * p.NF * d;               // M^{-1}, S_rr
    b += (5 + 2 * (size_t)p.s) * 3 * p.n * d;                 // q, q_new, R1, Z, Q, NL_i, L_i
    b += 5 * p.nt * d;                                        // g, x~, qhat, w, DG face fluxes
    if (c->precision == HDGDG_MIXED) {                        // FP32 S~, FP32 basis and work vector
        if (!matrix_free(c)) b += n_edges * 6 * (size_t)p.NF * p.NF * sizeof(float);
        b += ((size_t)p.m + (matrix_free(c) ? 4 : 2)) * p.nt * sizeof(float);   // basis and w (three, matrix-free)
    } else {
        b += ((size_t)p.m + 1) * p.nt * d;                    // FP64 Krylov basis
    }
    b += (reduction_scratch_doubles(p.m, (int)n_edges, (int)P) + mass_scratch_doubles() + 4 * (size_t)(p.m + 2) + 16) * d;
    b += 64 + sizeof(GmresCtl);                               // flags, GMRES control block
    if (c->local_precision == HDGDG_LOCAL_FP32) b += n_el * (size_t)p.NV * p.NV * sizeof(float);
    if (c->local_precision == HDGDG_LOCAL_BF16) b += tc_image_bytes((int)P);
    if (c->local_precision == HDGDG_LOCAL_BF16_SPLIT) b += tc_split_image_bytes((int)P);
    if (local_schur(c)) {   // (phi, phi) block of A^{-1}, 4 numbers per node, 2 P x P per instance
        b += (n_el * Np * Np + 4 * n_el * Np + 2 * B * Np) * d;   // FP64 or FP32 pairs: 8 bytes each
    } else if (c->local_precision == HDGDG_LOCAL_F32X2) {
        b += 2 * n_el * (size_t)p.NV * p.NV * sizeof(float);
    }
    if (c->precision == HDGDG_MIXED && c->residual_f32x2 && !matrix_free(c))
        b += n_edges * 6 * (size_t)p.NF * p.NF * sizeof(float);
    if (matrix_free(c)) {   // FP16 M^{-1} and scales, FP32 Schur operators, the operator's scratch
        b += n_edges * (size_t)p.NF * p.NF * sizeof(__half) + n_edges * sizeof(float);
        b += (n_el * Np * Np + 4 * n_el * Np + 2 * B * Np) * sizeof(float);
        b += 3 * p.nt * d;   // M^{-1} x and the two halves of S y
        b += n_edges * P * d;   // tau_hat as FP32 pairs
    }
    if (c->precision == HDGDG_MIXED && local_schur(c)) {   // FP32 stage values, phi_B and tau_hat
        b += (4 * p.n + n_edges * P) * sizeof(float);
    }
    b += 2 * (size_t)guess_order(c) * p.s * p.nt * d;         // previous stage solutions and products
    p.persistent = b;
    p.setup_temp = n_el * (size_t)p.NT * p.NT * d + n_edges * 7 * (size_t)p.NF * p.NF * d;
    if ((size_t)p.NV * 2 * p.NV * d > 200 * 1024)   // k >= 6: the local inverses' global workspace
        p.setup_temp += (n_el < 512 ? n_el : 512) * (size_t)p.NV * 2 * p.NV * d;
    return p;
}

// Host GLL tables: nodes by Newton on (1 - x^2) P_k'(x) = 0 in the form x P_k - P_{k-1} = 0
// (equivalent on the interior), weights 2 / (k (k+1) P_k^2), and the closed-form GLL
// differentiation matrix D_ij = P_k(x_i) / (P_k(x_j) (x_i - x_j)), D_00 = -k(k+1)/4,
// D_kk = k(k+1)/4, zero elsewhere on the diagonal.
void legendre(int k, double x, double* pk, double* pkm1) {
    double p0 = 1.0, p1 = x;
    if (k == 0) { *pk = 1.0; *pkm1 = 0.0; return; }
    for (int n = 1; n < k; ++n) {
        const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pk = p1;
    *pkm1 = p0;
}

void gll_tables(int k, double* x, double* w, double* D) {
    const int P = k + 1;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < P; ++i) {
        double xi = -std::cos(pi * i / k);
        if (i > 0 && i < k) {
            for (int it = 0; it < 100; ++it) {
                // Newton on f(x) = x P_k - P_{k-1}; f'(x) = (k+1) P_k (Legendre identity)
                double pk, pkm1;
                legendre(k, xi, &pk, &pkm1);
                const double dx = (xi * pk - pkm1) / ((k + 1.0) * pk);
                xi -= dx;
                if (std::fabs(dx) < 1e-16) break;
            }
        }
        x[i] = xi;
    }
    double Pk[kMaxP];
    for (int i = 0; i < P; ++i) {
        double pkm1;
        legendre(k, x[i], &Pk[i], &pkm1);
        w[i] = 2.0 / (k * (k + 1.0) * Pk[i] * Pk[i]);
    }
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
            double v = 0.0;
            if (i != j) v = Pk[i] / (Pk[j] * (x[i] - x[j]));
            else if (i == 0) v = -0.25 * k * (k + 1.0);
            else if (i == k) v = 0.25 * k * (k + 1.0);
            D[i * P + j] = v;
        }
}

Geom make_geom(const hdgdg_config* c, double* xi_out) {
    Geom g;
    std::memset(&g, 0, sizeof(g));
    g.N = c->n_side;
    g.P = c->degree_k + 1;
    g.Np = g.P * g.P;
    g.batch = c->batch > 0 ? c->batch : 1;
    g.n_el_inst = g.N * g.N;
    g.n_el = g.batch * g.n_el_inst;
    g.walls = c->boundary != HDGDG_PERIODIC ? 1 : 0;
    g.dirichlet = c->boundary == HDGDG_VORTEX ? 1 : 0;
    g.gacc = c->g;
    g.H0 = c->H0;
    for (int i = 0; i < 5; ++i) g.vortex[i] = c->bc_params[i];
    g.n_edges_inst = g.walls ? 2 * g.N * (g.N + 1) : 2 * g.n_el_inst;
    g.n_edges = g.batch * g.n_edges_inst;
    g.byN.set((unsigned)g.N);
    g.byN1.set((unsigned)g.N + 1u);
    g.by_el.set((unsigned)g.n_el_inst);
    g.by_edges.set((unsigned)g.n_edges_inst);
    g.dt_scale = nullptr;
    const double L = c->length > 0.0 ? c->length : 1.0;
    g.x0 = c->x0;
    g.h = L / g.N;
    g.two_over_h = 2.0 / g.h;
    g.J = 0.25 * g.h * g.h;
    double xi[kMaxP];
    gll_tables(c->degree_k, xi, g.w, g.D);
    for (int i = 0; i < g.P; ++i) g.xi[i] = xi[i];
    g.inv_w0 = 1.0 / g.w[0];
    for (int i = 0; i < g.P; ++i)
        for (int a = 0; a < g.P; ++a) g.Dhat[i * g.P + a] = (g.w[a] / g.w[i]) * g.D[a * g.P + i];
    if (xi_out)
        for (int i = 0; i < g.P; ++i) xi_out[i] = xi[i];
    return g;
}

void scheme_tables(int scheme, double A[kMaxStages][kMaxStages], double At[kMaxStages][kMaxStages],
                   double* b, double* bt, int* s) {
    std::memset(A, 0, sizeof(double) * kMaxStages * kMaxStages);
    std::memset(At, 0, sizeof(double) * kMaxStages * kMaxStages);
    if (scheme == HDGDG_ARS2) {
        // ARS(2,3,2), Ascher-Ruuth-Spiteri 1997: gamma = 1 - 1/sqrt 2, delta = -2 sqrt 2 / 3
        const double gm = 1.0 - 1.0 / std::sqrt(2.0), dl = -2.0 * std::sqrt(2.0) / 3.0;
        *s = 3;
        A[1][0] = gm;
        A[2][0] = dl;
        A[2][1] = 1.0 - dl;
        At[1][1] = gm;
        At[2][1] = 1.0 - gm;
        At[2][2] = gm;
        b[0] = 0.0; b[1] = 1.0 - gm; b[2] = gm;
        bt[0] = 0.0; bt[1] = 1.0 - gm; bt[2] = gm;
    } else {
        // ARS(4,4,3), Ascher-Ruuth-Spiteri 1997, implicit diagonal 1/2
        *s = 5;
        const double a[5][5] = {{0, 0, 0, 0, 0},
                                {1.0 / 2, 0, 0, 0, 0},
                                {11.0 / 18, 1.0 / 18, 0, 0, 0},
                                {5.0 / 6, -5.0 / 6, 1.0 / 2, 0, 0},
                                {1.0 / 4, 7.0 / 4, 3.0 / 4, -7.0 / 4, 0}};
        const double at[5][5] = {{0, 0, 0, 0, 0},
                                 {0, 1.0 / 2, 0, 0, 0},
                                 {0, 1.0 / 6, 1.0 / 2, 0, 0},
                                 {0, -1.0 / 2, 1.0 / 2, 1.0 / 2, 0},
                                 {0, 3.0 / 2, -3.0 / 2, 1.0 / 2, 1.0 / 2}};
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) { A[i][j] = a[i][j]; At[i][j] = at[i][j]; }
        for (int j = 0; j < 5; ++j) { b[j] = a[4][j]; bt[j] = at[4][j]; }
    }
}

}  // namespace

namespace hdgdg {
Geom host_geom(int N, int k) {
    hdgdg_config c{};
    c.n_side = N;
    c.degree_k = k;
    return make_geom(&c, nullptr);
}
}  // namespace hdgdg

// Two events bracketing a launch group of kernel class cls; slot >= 0 tags the groups of
// Arnoldi step `slot` of a GMRES cycle.
struct TimerPair {
    cudaEvent_t a, b;
    int cls, slot;
};

// NVTX range for profilers (a no-op unless one is attached): time steps, stage solves and
// GMRES restart cycles show up on their timelines.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    const double* g = nullptr;     // right-hand side the graph was captured for
    long long launches = 0;        // kernels per replay
    std::vector<TimerPair> timers; // event-record nodes of a graph captured with kernel timing on
};

// One time step captured as a CUDA graph with device-side solve control, keyed by the pointers and
// history lengths it was captured with (they change from step to step in a fixed cycle).
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    long long launches = 0;    // kernels captured (each restart-cycle body once)
    long long per_cycle = 0;   // kernels of one restart-cycle body
    int bodies = 0;            // restart-cycle bodies (one per implicit stage)
};

struct hdgdg_sim {
    hdgdg_config cfg;
    Plan plan;
    Geom g;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int s = 0;
    double A[kMaxStages][kMaxStages], At[kMaxStages][kMaxStages], b[kMaxStages], bt[kMaxStages];
    double a_ii = 0.0;
    // device memory
    std::vector<void*> allocs;
    double *phiB = nullptr, *tau = nullptr, *Ainv = nullptr, *Stil = nullptr, *Minv = nullptr, *Srr = nullptr;
    bool minv_pairs = false;   // residual_f32x2: M^{-1} rewritten in place as FP32 pairs after setup
    double* xhist[kMaxStages][6] = {};   // trace-solve guess: preconditioned solutions of the last
    double* yhist[kMaxStages][6] = {};   // steps per stage ([0] newest), their products S~ x~ (from
    int n_hist[kMaxStages] = {};         // the final true residual: g - r), and their count
    double dt_fingerprint = 0.0;  // sum_i (i + 1) dt_i of a batch with per-instance time steps
    float* Ainv32 = nullptr;      // HDGDG_LOCAL_FP32
    float *Ahi = nullptr, *Alo = nullptr;   // HDGDG_LOCAL_F32X2, dense
    double *Sphi = nullptr, *Saux = nullptr, *Seg = nullptr;   // Schur-complement local solves (8-byte
                                                                // values: FP64 or FP32 pairs)
    void* tc_image = nullptr;     // HDGDG_LOCAL_BF16: the shared operator's tensor-core tile
    LocalOps ops;
    int* Scol = nullptr;
    double *q = nullptr, *q_new = nullptr, *R1 = nullptr, *Z = nullptr, *Qs = nullptr;
    // per stage dt M^{-1} NL_i and Q_i - R1_i = dt a_ii M^{-1} L_i (the combinations divide by a_ii)
    double *NLs[kMaxStages] = {}, *Ls[kMaxStages] = {};
    double *gvec = nullptr, *xt = nullptr, *lam = nullptr, *w = nullptr, *V = nullptr, *fface = nullptr;
    float *Stil32 = nullptr, *V32 = nullptr, *w32 = nullptr;   // mixed precision only
    float* Stil_lo = nullptr;   // residual_f32x2: S~ = Stil32 + Stil_lo
    const EnsHost* ens = nullptr;   // an ensemble's super-handle: its group table (kernels walk every group)
    MfOps mf;                   // trace_operator = 1: the matrix-free operator's data
    int trace_tile = 0, trace_prefetch = 0;   // its autotuned element-pass tile (0: default)
    __half* Minv16 = nullptr;   // its block-Jacobi inverse: FP16 blocks ...
    float* Mscale = nullptr;    // ... and their power-of-two scales
    double *red = nullptr, *mred = nullptr, *dvals = nullptr;
    GmresCtl* ctl = nullptr;
    CycleGraph cycle_graph[4];   // [FP64 form, mixed form] x [timers off, on]
    std::vector<StepGraph> step_graphs;   // whole-step graphs (host_steps = 0, timers off)
    SolveCtl* sctl = nullptr;             // device-side control of the solve being replayed
    DevHist* dhist = nullptr;             // each stage's guess history, as the step graph reads it
    DevHist* hhist = nullptr;             // its pinned host copy, written before every replay
    double* dls = nullptr;                // the least-squares start's sums, choice and coefficients
    // mixed form with the Schur-complement local solves: the DG residual's FP32 copies (phi_B,
    // tau) and the recovery's FP32 stage values; the face fluxes then sit in fface as FP32
    float* Qs32 = nullptr;
    float* phiB32 = nullptr;
    float* tau32 = nullptr;
    StepStats* sstats = nullptr;          // counters of the replayed step
    cudaStream_t body_stream = nullptr;   // captures the restart-cycle bodies of the conditional nodes
    // the step graph's branch beside the recovery: each stage's guess-history store (fork and join
    // events per stage)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_ev[kMaxStages] = {}, join_ev[kMaxStages] = {};
    std::vector<TimerPair>* capture_sink = nullptr;   // timers of the graph being captured
    unsigned* flags = nullptr;
    double* hbuf = nullptr;   // pinned host scratch
    // run state
    bool have_state = false;
    double t = 0.0;
    hdgdg_stats stats{};
    // per-kernel-class timers
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<TimerPair> pending;
    double kt_ms[HDGDG_KT_COUNT] = {};
    long long kt_n[HDGDG_KT_COUNT] = {};
};

namespace {

hdgdg_status fail(hdgdg_sim* s, hdgdg_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    return st;
}

#define CU(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(sim, HDGDG_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                     \
    } while (0)

template <typename T>
hdgdg_status dalloc(hdgdg_sim* sim, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(sim, HDGDG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    sim->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return HDGDG_OK;
}

#define TRY(x)                               \
    do {                                     \
        hdgdg_status st_ = (x);              \
        if (st_ != HDGDG_OK) return st_;     \
    } while (0)

// Slots of the small device array dvals
inline double* dv_h1(hdgdg_sim* s) { return s->dvals; }
inline double* dv_h2(hdgdg_sim* s) { return s->dvals + (s->plan.m + 2); }
// device error word of the pipelined SpMV (a bounded wait ran out)
inline int* spmv_error(hdgdg_sim* s) { return reinterpret_cast<int*>(s->flags) + 3; }
inline double* dv_nrm(hdgdg_sim* s) { return s->dvals + 2 * (s->plan.m + 2); }
inline double* dv_guess(hdgdg_sim* s) { return s->dvals + 3 * (s->plan.m + 2) + 8; }   // 7 slots

cudaEvent_t take_event(hdgdg_sim* sim) {
    if (!sim->ev_pool.empty()) {
        cudaEvent_t e = sim->ev_pool.back();
        sim->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket a launch group of class cls with events (no-op unless timing is on).  slot >= 0
// tags groups enqueued speculatively in a GMRES cycle: the ones at or after the cycle's
// actual length returned at once and are dropped when the timers are read.
struct TimedGroup {
    hdgdg_sim* sim;
    int cls, slot;
    cudaEvent_t a = nullptr;
    TimedGroup(hdgdg_sim* s, int c, int sl = -1) : sim(s), cls(c), slot(sl) {
        if (sim->timing && (a = take_event(sim))) record(a);
    }
    // Inside a stream capture a plain event record only orders the capture; an external record
    // becomes a graph node that records the event at every replay.
    void record(cudaEvent_t e) const {
        if (sim->capture_sink) cudaEventRecordWithFlags(e, sim->stream, cudaEventRecordExternal);
        else cudaEventRecord(e, sim->stream);
    }
    ~TimedGroup() {
        if (!a) return;
        cudaEvent_t b = take_event(sim);
        if (!b) { sim->ev_pool.push_back(a); return; }
        record(b);
        // groups recorded while a GMRES cycle is captured belong to that graph and are read
        // after each of its replays
        (sim->capture_sink ? sim->capture_sink : &sim->pending)->push_back({a, b, cls, slot});
    }
};

void flush_timers(hdgdg_sim* sim, int slot_limit = 1 << 30) {
    for (auto& p : sim->pending) {
        float ms = 0.f;
        if (p.slot < slot_limit) {
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                sim->kt_ms[p.cls] += ms;
                sim->kt_n[p.cls] += 1;
            } else {
                cudaGetLastError();   // a timer that could not be read is skipped, not an error
            }
        }
        sim->ev_pool.push_back(p.a);
        sim->ev_pool.push_back(p.b);
    }
    sim->pending.clear();
}

// Add a replayed graph's timers (groups of Arnoldi steps at or after slot_limit returned at once).
void read_graph_timers(hdgdg_sim* sim, const CycleGraph& cg, int slot_limit) {
    for (const auto& p : cg.timers) {
        float ms = 0.f;
        if (p.slot >= slot_limit) continue;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            sim->kt_ms[p.cls] += ms;
            sim->kt_n[p.cls] += 1;
        } else {
            cudaGetLastError();
        }
    }
}

void drop_graph(hdgdg_sim* sim, CycleGraph& cg) {
    if (cg.exec) cudaGraphExecDestroy(cg.exec);
    cg.exec = nullptr;
    for (const auto& p : cg.timers) {
        sim->ev_pool.push_back(p.a);
        sim->ev_pool.push_back(p.b);
    }
    cg.timers.clear();
}

hdgdg_status sync(hdgdg_sim* sim, int slot_limit = 1 << 30) {
    CU(cudaStreamSynchronize(sim->stream));
    flush_timers(sim, slot_limit);
    return HDGDG_OK;
}

// ||v||^2 into dv_nrm, copied to host hbuf[0]
hdgdg_status norm2_to_host(hdgdg_sim* sim, const double* v, double* out) {
    CU(launch_multidot(v, 0, 1, v, sim->plan.nt, sim->red, dv_nrm(sim), sim->stream));
    CU(cudaMemcpyAsync(sim->hbuf, dv_nrm(sim), sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    TRY(sync(sim));
    *out = sim->hbuf[0];
    return HDGDG_OK;
}

// Lift factor of the local solves: -B qhat = beta tau qhat on the boundary nodes, beta = dt a_ii (2/h)/w_0
double beta_of(const hdgdg_sim* sim) { return sim->cfg.dt * sim->a_ii * sim->g.two_over_h * sim->g.inv_w0; }

// A restart cycle that cannot halve a true residual already below kStagnation * ||g|| has reached
// the rounding floor of the FP64 residual: the solve accepts it.
constexpr double kStagnationFloor = 1e-12;
// Extrapolation coefficients of the initial guess, order q = 1..6: x_0 = sum_j c[q][j] x_{n-1-j}.
constexpr double kGuessCoef[7][6] = {{0, 0, 0, 0, 0, 0},     {1, 0, 0, 0, 0, 0},     {2, -1, 0, 0, 0, 0},
                                     {3, -3, 1, 0, 0, 0},    {4, -6, 4, -1, 0, 0},   {5, -10, 10, -5, 1, 0},
                                     {6, -15, 20, -15, 6, -1}};
inline double* dv_exact(hdgdg_sim* s) { return s->dvals + 3 * (s->plan.m + 2) + 15; }

// One restart cycle on stream st: m Arnoldi steps (the ones after the cycle's stop return at
// once), the correction, the true residual and its squared norm in dv_nrm; readback: also copy
// the norm and the control flags to the pinned host buffer (the host-driven loop reads them).
template <typename T>
cudaError_t cycle_enqueue(hdgdg_sim* sim, const double* g, cudaStream_t st, bool readback) {
    constexpr bool kMixed = sizeof(T) == sizeof(float);
    const size_t n = sim->plan.nt;
    const int m = sim->plan.m;
    T* V = nullptr;
    T* w = nullptr;
    const T* St = nullptr;
    if constexpr (kMixed) { V = sim->V32; w = sim->w32; St = sim->Stil32; }
    else { V = sim->V; w = sim->w; St = sim->Stil; }
    GmresCtl* ctl = sim->ctl;
    const int* done = &ctl->done;
    // The fused matrix-free product adds into its output, so the products alternate between two
    // vectors (w32 holds both): the cycle's first launch zeroes the first, and iteration j's
    // Gram-Schmidt tail zeroes the one product j + 1 adds into.
    const bool fused = kMixed && matrix_free(&sim->cfg) && !sim->ens;
    cudaError_t e = launch_gmres_cycle_init(ctl, dv_nrm(sim), st);
    if (e == cudaSuccess) {
        if constexpr (kMixed) e = launch_scale_by_rnorm(sim->w, dv_nrm(sim), V, n, st, fused ? w : nullptr);
        else e = launch_scale_by_rnorm(sim->w, dv_nrm(sim), V, n, st);
    }
    T* const w_base = w;
    // FP32 matrix-free cycles with Gram-Schmidt twice: the second pass is delayed into the next
    // step (launch_dcgs_fused), whose product is taken of w1 (always in w32's first vector); the
    // products then alternate between the second and third vectors, each zeroed one step ahead
    const bool delayed = fused && sim->cfg.krylov_ortho != 1;
    if constexpr (kMixed) {
        if (delayed && e == cudaSuccess) e = cudaMemsetAsync(w_base + n, 0, n * sizeof(T), st);
        for (int j = 0; delayed && j < m && e == cudaSuccess; ++j) {
            T* const A = w_base;
            T* const Tj = w_base + (size_t)(1 + (j + 1) % 2) * n;   // this step's product (j >= 1)
            T* const Tn = w_base + (size_t)(1 + j % 2) * n;         // the next step's
            {
                TimedGroup tg(sim, HDGDG_KT_SPMV, j);
                e = launch_mf_inner(sim->g, sim->mf, j == 0 ? V : A, j == 0 ? A : Tj, beta_of(sim), st, done, true);
            }
            TimedGroup tg(sim, HDGDG_KT_ORTHO, j);
            if (e == cudaSuccess)
                e = j == 0 ? launch_multidot(V, n, 1, A, n, sim->red, dv_h1(sim), st, done)
                           : launch_dcgs_fused(V, n, j, dv_h2(sim), dv_nrm(sim) + 1, ctl, A, Tj, V + (size_t)j * n, Tn,
                                               n, sim->red, dv_h1(sim), st, done);
            if (e == cudaSuccess)
                e = launch_cgs2_update(V, n, j + 1, dv_h1(sim), A, n, sim->red, dv_h2(sim), dv_nrm(sim) + 2,
                                       dv_nrm(sim) + 1, ctl, j, m, st, done);
        }
    }
    for (int j = 0; !delayed && j < m && e == cudaSuccess; ++j) {
        const T* Vj = V + (size_t)j * n;
        if (fused) w = w_base + (size_t)(j % 2) * n;
        {
            TimedGroup tg(sim, HDGDG_KT_SPMV, j);
            if constexpr (kMixed) {
                if (sim->ens) e = launch_ens_mf_inner(*sim->ens, sim->mf, n, Vj, w, st, done);
                else if (fused) e = launch_mf_inner(sim->g, sim->mf, Vj, w, beta_of(sim), st, done, true);
                else
                    e = launch_spmv_pre(sim->g, St, sim->Scol, Vj, w, st, done,
                                        sim->cfg.spmv_kernel == 1 ? spmv_error(sim) : nullptr);
            } else
                e = launch_spmv_pre(sim->g, St, sim->Scol, Vj, w, st, done);
        }
        TimedGroup tg(sim, HDGDG_KT_ORTHO, j);
        if (e == cudaSuccess) e = launch_multidot(V, n, j + 1, w, n, sim->red, dv_h1(sim), st, done);
        if (e == cudaSuccess) {   // second pass, norm, Hessenberg column j and stop test
            if constexpr (kMixed)
                e = launch_cgs2_tail(V, n, j + 1, dv_h1(sim), w, n, sim->red, dv_h2(sim), dv_nrm(sim) + 2,
                                     dv_nrm(sim) + 1, V + (size_t)(j + 1) * n, ctl, j, m,
                                     sim->cfg.krylov_ortho != 1, st, done,
                                     fused ? w_base + (size_t)((j + 1) % 2) * n : nullptr);
            else
                e = launch_cgs2_tail(V, n, j + 1, dv_h1(sim), w, n, sim->red, dv_h2(sim), dv_nrm(sim) + 2,
                                     dv_nrm(sim) + 1, V + (size_t)(j + 1) * n, ctl, j, m, true, st, done);
        }
    }
    TimedGroup tg_end(sim, HDGDG_KT_RESIDUAL);
    if (e == cudaSuccess) e = launch_gmres_update(V, n, ctl, sim->xt, n, st);
    // the true residual w = g - S~ x~ that ends the cycle, and ||w||^2
    if (kMixed && matrix_free(&sim->cfg)) {   // matrix-free in FP32-pair arithmetic, then the norm
        if (e == cudaSuccess) {
            if (sim->ens) {
                e = launch_ens_mf_residual(*sim->ens, sim->mf, n, sim->xt, g, sim->w, st);
                if (e == cudaSuccess) e = launch_multidot(sim->w, 0, 1, sim->w, n, sim->red, dv_nrm(sim), st);
            } else {   // the last pass also forms ||w||^2
                e = launch_mf_residual(sim->g, sim->mf, sim->xt, g, sim->w, beta_of(sim), st, sim->red, dv_nrm(sim));
            }
        }
    } else if (kMixed && sim->Stil_lo) {   // one fused FP32-pair pass
        if (e == cudaSuccess)
            e = launch_residual_norm_x2(sim->g, sim->Stil32, sim->Stil_lo, sim->Scol, sim->xt, g, sim->w,
                                        sim->red, dv_nrm(sim), st);
    } else {
        if (e == cudaSuccess) e = launch_spmv_pre(sim->g, sim->Stil, sim->Scol, sim->xt, sim->w, st);
        CombineTerms t{};
        t.n = 1;
        t.X[0] = sim->w;
        t.c[0] = -1.0;
        if (e == cudaSuccess) e = launch_combine(n, g, t, sim->w, nullptr, st);
        if (e == cudaSuccess) e = launch_multidot(sim->w, 0, 1, sim->w, n, sim->red, dv_nrm(sim), st);
    }
    if (readback && e == cudaSuccess)
        e = cudaMemcpyAsync(sim->hbuf, dv_nrm(sim), sizeof(double), cudaMemcpyDeviceToHost, st);
    if (readback && e == cudaSuccess)
        e = cudaMemcpyAsync(sim->hbuf + 1, &ctl->done, 5 * sizeof(int), cudaMemcpyDeviceToHost, st);
    return e;
}

// Right-preconditioned GMRES(m) on S~ x~ = g with classical Gram-Schmidt applied twice, then
// qhat = M^{-1} x~.  The Givens rotations, the residual estimate and the stop test run on the
// device (GmresCtl), so a whole restart cycle is queued at once and the host waits once per
// cycle: the loop kernels after the cycle's last useful iteration return immediately.
// T = double: the FP64 form.  T = float (mixed form): the cycle runs on the FP32 copy of S~
// and FP32 basis vectors; every cycle starts from the true residual r = g - S~ x~ computed in
// FP64 and adds its correction to the FP64 x~ (iterative refinement).
template <typename T>
hdgdg_status gmres_solve(hdgdg_sim* sim, const double* g, double* qhat, int* iters, double* relres,
                         int stage) {
    constexpr bool kMixed = sizeof(T) == sizeof(float);
    const size_t n = sim->plan.nt;
    const double rtol = sim->cfg.krylov_rtol > 0.0 ? sim->cfg.krylov_rtol : (kMixed ? 1e-9 : 1e-15);
    const int maxit = sim->cfg.krylov_maxit > 0 ? sim->cfg.krylov_maxit : 2000;
    // Mixed form: an FP32 cycle stops once it has reduced its starting residual 1e6 times.
    const double inner_rel = kMixed ? 1e-6 : 0.0;
    constexpr double kStagnation = kStagnationFloor;
    cudaStream_t st = sim->stream;
    GmresCtl* ctl = sim->ctl;
    *iters = 0;
    // Initial guess: the extrapolation in time of the stage's previous solutions, at the order
    // (or zero) whose residual is smallest.  One pass over g and the stored products S~ x~_{n-j}
    // gives ||g||^2 and every candidate's residual norm; no matrix product is needed.
    const auto& coef = kGuessCoef;
    const int avail = stage >= 0 ? std::min(guess_order(&sim->cfg), sim->n_hist[stage]) : 0;
    double cand[7] = {0, 0, 0, 0, 0, 0, 0};
    const bool ls = kMixed && sim->cfg.krylov_guess_ls && avail > 0;   // the least-squares start
    double alpha[6] = {0, 0, 0, 0, 0, 0};
    if (ls) {
        GuessTerms gt{};
        gt.nq = avail;
        for (int j = 0; j < avail; ++j) gt.y[j] = sim->yhist[stage][j];
        {
            TimedGroup tg(sim, HDGDG_KT_GUESS);
            CU(launch_guess_gram(n, g, gt, sim->red, sim->dls, st));
            CU(launch_ls_solve(sim->dls, avail, st));
            CU(cudaMemcpyAsync(sim->hbuf, sim->dls + 32, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        TRY(sync(sim));
        cand[0] = sim->hbuf[0];
        cand[1] = sim->hbuf[1];
        std::memcpy(alpha, sim->hbuf + 2, sizeof(alpha));
    } else if (avail > 0) {
        GuessTerms gt{};
        gt.nq = avail;
        for (int j = 0; j < avail; ++j) gt.y[j] = sim->yhist[stage][j];
        std::memcpy(gt.c, coef, sizeof(coef));
        {   // (the group ends before the host waits: the wait is not GPU time)
            TimedGroup tg(sim, HDGDG_KT_GUESS);
            CU(launch_guess_norms(n, g, gt, sim->red, dv_guess(sim), st, kMixed));
            CU(cudaMemcpyAsync(sim->hbuf, dv_guess(sim), (avail + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        TRY(sync(sim));
        std::memcpy(cand, sim->hbuf, (avail + 1) * sizeof(double));
    } else {
        TRY(norm2_to_host(sim, g, &cand[0]));
    }
    const double bn2 = cand[0];
    if (!std::isfinite(bn2)) return fail(sim, HDGDG_ENONFINITE, "non-finite trace right-hand side");
    if (bn2 == 0.0) {
        CU(cudaMemsetAsync(qhat, 0, n * sizeof(double), st));
        *relres = 0.0;
        return HDGDG_OK;
    }
    const double bnorm = std::sqrt(bn2), tol = rtol * bnorm;
    int guess = 0;
    for (int q = 1; q <= (ls ? 1 : avail); ++q)
        if (std::isfinite(cand[q]) && cand[q] < cand[guess]) guess = q;
    sim->stats.last_guess_order = guess;
    const double rnorm0 = std::sqrt(cand[guess]);
    double rnorm = rnorm0;
    {
        TimedGroup tg_guess(sim, HDGDG_KT_GUESS);
        if (guess == 0) {
            CU(cudaMemsetAsync(sim->xt, 0, n * sizeof(double), st));
            CU(cudaMemcpyAsync(sim->w, g, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if (avail > 0)   // ||g||^2 for the cycle's first basis vector (norm2_to_host left it otherwise)
                CU(cudaMemcpyAsync(dv_nrm(sim), ls ? sim->dls + 32 : dv_guess(sim), sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
        } else if (ls) {
            // x0 = sum_j alpha_j x_{n-j} and r0 = g - sum_j alpha_j S~ x~_{n-j}, the graph's sums
            CombineTerms t{};
            for (int j = 0; j < avail; ++j) {
                t.X[t.n] = sim->xhist[stage][j];
                t.c[t.n++] = alpha[j] - (j == 0 ? 1.0 : 0.0);
            }
            CU(launch_combine(n, sim->xhist[stage][0], t, sim->xt, nullptr, st));
            CombineTerms r{};
            for (int j = 0; j < avail; ++j) {
                r.X[r.n] = sim->yhist[stage][j];
                r.c[r.n++] = -alpha[j];
            }
            CU(launch_combine(n, g, r, sim->w, nullptr, st));
            CU(launch_multidot(sim->w, 0, 1, sim->w, n, sim->red, dv_nrm(sim), st));   // the exact start norm
        } else {
            // x0 = sum_j c_j x_{n-j}: the extrapolation polynomial through the last `guess` solutions
            CombineTerms t{};
            for (int j = 0; j < guess; ++j) {
                t.X[t.n] = sim->xhist[stage][j];
                t.c[t.n++] = coef[guess][j] - (j == 0 ? 1.0 : 0.0);   // base x_{n-1} counted once
            }
            CU(launch_combine(n, sim->xhist[stage][0], t, sim->xt, nullptr, st));
            // r0 = g - S~ x0 = g - sum_j c_j (S~ x~_{n-j}): S~ is linear, and each S~ x~_{n-j} is
            // known from the true residual that ended that step's solve -- no product needed
            CombineTerms r{};
            for (int j = 0; j < guess; ++j) {
                r.X[r.n] = sim->yhist[stage][j];
                r.c[r.n++] = -coef[guess][j];
            }
            CU(launch_combine(n, g, r, sim->w, nullptr, st));
            if constexpr (kMixed)   // the candidates were FP32-pair estimates: the cycle's start norm exactly
                CU(launch_multidot(sim->w, 0, 1, sim->w, n, sim->red, dv_nrm(sim), st));
            else
                CU(cudaMemcpyAsync(dv_nrm(sim), dv_guess(sim) + guess, sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
    }
    CU(launch_gmres_solve_init(ctl, tol, inner_rel, maxit, st));
    int total = 0;
    // One restart cycle: m Arnoldi steps (the ones after the cycle's stop return at once), the
    // correction, the FP64 true residual and its read-back.  Without kernel timing the cycle is
    // captured once per handle and form as a CUDA graph and replayed.
    auto enqueue_cycle = [&]() -> cudaError_t { return cycle_enqueue<T>(sim, g, st, true); };
    // one graph per form, captured with or without the kernel-class timers (event-record nodes)
    CycleGraph& cg = sim->cycle_graph[(kMixed ? 1 : 0) + (sim->timing ? 2 : 0)];
    while (rnorm > tol) {
        if (cg.exec && cg.g != g) drop_graph(sim, cg);
        if (!cg.exec) {
            const long long l0 = launches_total();
            if (sim->timing) sim->capture_sink = &cg.timers;
            CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e = enqueue_cycle();
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            sim->capture_sink = nullptr;
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                drop_graph(sim, cg);
                return fail(sim, HDGDG_ECUDA, "capturing the GMRES cycle failed: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            const cudaError_t e3 = cudaGraphInstantiate(&cg.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                cg.exec = nullptr;
                drop_graph(sim, cg);
                return fail(sim, HDGDG_ECUDA, "GMRES cycle graph: %s", cudaGetErrorString(e3));
            }
            cg.g = g;
            cg.launches = launches_total() - l0;
            count_launches((int)-cg.launches);   // counted again at every replay below
        }
        NvtxRange nv_cycle("gmres_cycle");
        CU(cudaGraphLaunch(cg.exec, st));
        count_launches((int)cg.launches);
        CU(cudaStreamSynchronize(st));
        int cf[5];   // done, jend, total, maxit, status
        std::memcpy(cf, sim->hbuf + 1, sizeof(cf));
        flush_timers(sim, cf[1]);
        if (sim->timing) read_graph_timers(sim, cg, cf[1]);
        total = cf[2];
        if (cf[4] != 0)
            return fail(sim, HDGDG_ENONFINITE, "non-finite GMRES residual estimate at iteration %d", total);
        const double rn2 = sim->hbuf[0];
        if (!std::isfinite(rn2)) return fail(sim, HDGDG_ENONFINITE, "non-finite GMRES residual");
        const double prev = rnorm;
        rnorm = std::sqrt(rn2);
        if (rnorm <= tol) break;
        if (rnorm <= kStagnation * bnorm && rnorm > 0.5 * prev) break;
        if (total >= maxit) {
            *iters = total;
            *relres = rnorm / bnorm;
            sim->stats.last_krylov_iterations = total;
            sim->stats.last_rel_residual = *relres;
            return fail(sim, HDGDG_ENOTCONVERGED, "GMRES: relative residual %.3e > %.3e after %d iterations",
                        rnorm / bnorm, rtol, total);
        }
    }
    {
        TimedGroup tg(sim, HDGDG_KT_PRECOND);
        if (kMixed && matrix_free(&sim->cfg)) CU(launch_mf_back(sim->g, sim->mf.Minv, sim->xt, qhat, st));
        else CU(launch_block_diag(sim->g, sim->Minv, sim->xt, qhat, st, sim->minv_pairs));
    }
    const int order = guess_order(&sim->cfg);
    if (stage >= 0 && order > 0) {   // keep x~ and S~ x~ = g - r for the next steps' guesses
        TimedGroup tg(sim, HDGDG_KT_GUESS);
        double* ox = sim->xhist[stage][order - 1];
        double* oy = sim->yhist[stage][order - 1];
        for (int j = order - 1; j > 0; --j) {
            sim->xhist[stage][j] = sim->xhist[stage][j - 1];
            sim->yhist[stage][j] = sim->yhist[stage][j - 1];
        }
        sim->xhist[stage][0] = ox;
        sim->yhist[stage][0] = oy;
        CU(cudaMemcpyAsync(ox, sim->xt, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CombineTerms r{};   // sim->w holds the final true residual g - S~ x~
        r.n = 1;
        r.X[0] = sim->w;
        r.c[0] = -1.0;
        CU(launch_combine(n, g, r, oy, nullptr, st));
        sim->n_hist[stage] = std::min(sim->n_hist[stage] + 1, order);
    }
    *iters = total;
    *relres = rnorm / bnorm;
    sim->stats.last_krylov_iterations = total;
    sim->stats.last_rel_residual = *relres;
    sim->stats.krylov_iterations += total;
    return HDGDG_OK;
}


// Whether an implicit stage's condensation forms R1 from its terms (launch_condense's src): the
// FP32-pair Schur kernels, whose time goes to FP32 work and latency, absorb the combination's
// streams; the FP64 ones are bound by the FP64 pipe, which its FMAs would lengthen.
bool r1_fused(const hdgdg_sim* sim, const CombineTerms& t) {
    return sim->ops.schur && sim->ops.kind == 3 && t.n <= kR1FusedTerms;
}

// One implicit stage: R1 (device) -> Q, Lst = Q - R1 = dt a_ii M^{-1} L (device); qhat left in
// sim->lam.  src: R1 is formed by the condensation from these terms (launch_condense) instead of read.
hdgdg_status stage_solve_dev(hdgdg_sim* sim, const double* R1, double* Q, double* Lst, int* its,
                             double t_stage = 0.0, int stage = -1, float* Q32 = nullptr,
                             const R1Source* src = nullptr) {
    NvtxRange nv("stage_solve");
    double rr;
    {
        TimedGroup tg(sim, HDGDG_KT_CONDENSE);
        CU(launch_condense(sim->g, sim->ops, R1, sim->phiB, sim->tau, sim->Z, sim->gvec, sim->stream, t_stage,
                           src));
    }
    if (sim->cfg.precision == HDGDG_MIXED) TRY(gmres_solve<float>(sim, sim->gvec, sim->lam, its, &rr, stage));
    else TRY(gmres_solve<double>(sim, sim->gvec, sim->lam, its, &rr, stage));
    {
        TimedGroup tg(sim, HDGDG_KT_RECOVER);
        CU(launch_recover(sim->g, sim->ops, sim->Z, R1, sim->tau, sim->lam, beta_of(sim), 1.0,
                          Q, Lst, sim->stream, Q32));
    }
    return HDGDG_OK;
}

// The nonlinear DG residual of stage value Qi into out.  stage_value: Qi came from this step's
// recovery (with the FP32 copies, its FP32 copy in Qs32 is the one written).
// fin: the step's final update formed by the element pass (dg_final_fusable).
cudaError_t dg_nl_enqueue(hdgdg_sim* sim, const double* Qi, bool stage_value, double* out, cudaStream_t st,
                          double t, const FinalSource* fin = nullptr) {
    if (fin && !(sim->cfg.precision == HDGDG_MIXED && sim->Qs32 && stage_value && !sim->ens &&
                 sim->cfg.dg_precision != 1))
        return cudaErrorInvalidValue;
    if (sim->ens) return launch_ens_dg_nl_f32(*sim->ens, Qi, sim->fface, out, st);
    if (sim->cfg.dg_precision == 1)
        return launch_dg_nl_bf16(sim->g, Qi, sim->phiB, sim->tau, sim->cfg.dt, sim->fface, out, st, t);
    if (sim->cfg.precision == HDGDG_MIXED && sim->Qs32)
        return launch_dg_nl_f32io(sim->g, Qi, stage_value ? sim->Qs32 : nullptr, sim->phiB32, sim->tau32, sim->cfg.dt,
                                  reinterpret_cast<float*>(sim->fface), out, st, t, fin);
    if (sim->cfg.precision == HDGDG_MIXED)
        return launch_dg_nl_f32(sim->g, Qi, sim->phiB, sim->tau, sim->cfg.dt, sim->fface, out, st, t);
    return launch_dg_nl(sim->g, Qi, sim->phiB, sim->tau, sim->cfg.dt, sim->fface, out, st, t);
}

// ---- whole-step graphs ------------------------------------------------------------------------
// The trace solve of gmres_solve with every host decision moved to the device (kernels_ctl.cu),
// enqueued on st while a whole time step is being captured: the candidate norms, the choice of the
// start, the restart cycles inside a conditional while node (body captured on the handle's body
// stream), the counters, the back-transformation and the history copy into the slot that becomes
// the newest when the host rotates the history after the step.
// defer_hist: the history store is left to the caller (step_enqueue_graph's side branch).
template <typename T>
cudaError_t solve_enqueue_graph(hdgdg_sim* sim, const double* g, double* qhat, int stage, cudaStream_t st,
                                StepGraph& sg, bool defer_hist = false) {
    constexpr bool kMixed = sizeof(T) == sizeof(float);
    const size_t n = sim->plan.nt;
    const double rtol = sim->cfg.krylov_rtol > 0.0 ? sim->cfg.krylov_rtol : (kMixed ? 1e-9 : 1e-15);
    const int maxit = sim->cfg.krylov_maxit > 0 ? sim->cfg.krylov_maxit : 2000;
    const double inner_rel = kMixed ? 1e-6 : 0.0;
    const int order = guess_order(&sim->cfg);
    const bool history = stage >= 0 && order > 0;
    cudaError_t e = cudaSuccess;
    if (history && kMixed && sim->cfg.krylov_guess_ls) {   // the least-squares start, from the device table
        const DevHist* dh = sim->dhist + stage;
        e = launch_multidot(g, 0, 1, g, n, sim->red, sim->dls + 32, st, &dh->has_history);
        if (e == cudaSuccess) e = launch_guess_gram_dev(n, g, dh, sim->red, sim->dls, st);
        if (e == cudaSuccess)
            e = launch_ls_start_dev(n, g, dh, sim->dls, rtol, inner_rel, maxit, sim->ctl, sim->sctl, sim->sstats,
                                    dv_nrm(sim), sim->xt, sim->w, st);
    } else if (history) {   // the history's length and pointers come from the stage's device table
        const DevHist* dh = sim->dhist + stage;
        // ||g||^2 alone when the history is empty (the kernel returns at once otherwise), else the
        // candidates' norms
        e = launch_multidot(g, 0, 1, g, n, sim->red, dv_guess(sim), st, &dh->has_history);
        if (e == cudaSuccess) e = launch_guess_norms_dev(n, g, dh, kGuessCoef, sim->red, dv_guess(sim), st, kMixed);
        if (e == cudaSuccess)
            e = launch_solve_begin_dev(dv_guess(sim), dh, rtol, inner_rel, maxit, sim->ctl, sim->sctl, sim->sstats,
                                       dv_nrm(sim), st);
        if (e == cudaSuccess) e = launch_guess_apply_dev(n, g, dh, kGuessCoef, sim->sctl, sim->xt, sim->w, st);
    } else {
        e = launch_multidot(g, 0, 1, g, n, sim->red, dv_guess(sim), st);
        if (e == cudaSuccess)
            e = launch_solve_begin(dv_guess(sim), 0, rtol, inner_rel, maxit, sim->ctl, sim->sctl, sim->sstats,
                                   dv_nrm(sim), st);
        GuessHistory hist{};
        std::memcpy(hist.c, kGuessCoef, sizeof(kGuessCoef));
        if (e == cudaSuccess) e = launch_guess_apply(n, g, hist, sim->sctl, sim->xt, sim->w, st);
    }
    if (kMixed && e == cudaSuccess)   // the exact start norm of an extrapolated start
        e = launch_multidot(sim->w, 0, 1, sim->w, n, sim->red, dv_exact(sim), st);
    // restart cycles while the true residual is above the tolerance
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle loop = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, graph, 0, 0);
    if (e == cudaSuccess)
        e = launch_loop_begin(dv_nrm(sim), dv_exact(sim), kMixed ? 1 : 0, sim->sctl, sim->sstats, loop, st);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(sim->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const long long l0 = launches_total();
            cudaError_t eb = cycle_enqueue<T>(sim, g, sim->body_stream, false);
            if (eb == cudaSuccess)
                eb = launch_cycle_end(dv_nrm(sim), sim->ctl, sim->sctl, sim->sstats, kStagnationFloor, loop,
                                      sim->body_stream);
            sg.per_cycle = launches_total() - l0;
            sg.bodies += 1;
            cudaGraph_t captured = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(sim->body_stream, &captured);
            e = eb != cudaSuccess ? eb : ee;
        }
    }
    if (e == cudaSuccess) e = launch_solve_end(sim->ctl, sim->sctl, sim->sstats, st);
    if (e == cudaSuccess) {
        if (sim->ens) e = launch_ens_mf_back(*sim->ens, sim->xt, qhat, st);
        else if (kMixed && matrix_free(&sim->cfg)) e = launch_mf_back(sim->g, sim->mf.Minv, sim->xt, qhat, st);
        else e = launch_block_diag(sim->g, sim->Minv, sim->xt, qhat, st, sim->minv_pairs);
    }
    if (e == cudaSuccess && history && !defer_hist)   // x~ and S~ x~ = g - r into the slot that becomes newest
        e = launch_hist_store_dev(n, sim->xt, g, sim->w, sim->dhist + stage, st);
    return e;
}

// One implicit time step (Algorithm 1) enqueued for capture: the host-driven step's launches,
// with the trace solves of solve_enqueue_graph and no host waits; the step's flags and counters
// are copied to the pinned host buffer at its end.
cudaError_t step_enqueue_graph(hdgdg_sim* sim, cudaStream_t st, StepGraph& sg) {
    const size_t n3 = 3 * sim->plan.n;
    cudaError_t e = cudaMemsetAsync(sim->sstats, 0, sizeof(StepStats), st);
    // the final update's terms, in their order; where the last stage's DG residual is one of them
    // and the mixed form's FP32-input element pass computes it, that pass forms q_new itself
    CombineTerms tf{};
    int slot = -1;
    for (int i = 0; i < sim->s; ++i) {
        if (sim->b[i] != 0.0 && !sim->cfg.linear_only) {
            if (i == sim->s - 1) slot = tf.n;
            tf.X[tf.n] = sim->NLs[i];
            tf.c[tf.n++] = sim->b[i];
        }
        if (sim->bt[i] != 0.0) { tf.X[tf.n] = sim->Ls[i]; tf.c[tf.n++] = sim->bt[i] / sim->a_ii; }
    }
    const bool fuse_final = slot >= 0 && tf.n <= kFinalTerms && !sim->ens && sim->cfg.precision == HDGDG_MIXED &&
                            sim->Qs32 && sim->cfg.dg_precision != 1 && sim->At[sim->s - 1][sim->s - 1] != 0.0;
    // each stage's history store reads x~, g and r, which nothing overwrites before the next
    // stage's condensation: it runs on a branch beside the recovery and the DG residual
    const bool branch = !sim->ens && sim->side_stream && guess_order(&sim->cfg) > 0;
    int pending = -1;   // the stage whose store has not joined yet
    for (int i = 0; i < sim->s && e == cudaSuccess; ++i) {
        const double* Qi = sim->q;
        if (sim->At[i][i] != 0.0) {
            if (pending >= 0) {
                e = cudaStreamWaitEvent(st, sim->join_ev[pending], 0);
                pending = -1;
                if (e != cudaSuccess) break;
            }
            CombineTerms t{};
            for (int j = 0; j < i; ++j) {
                if (sim->A[i][j] != 0.0 && !sim->cfg.linear_only) { t.X[t.n] = sim->NLs[j]; t.c[t.n++] = sim->A[i][j]; }
                if (sim->At[i][j] != 0.0) { t.X[t.n] = sim->Ls[j]; t.c[t.n++] = sim->At[i][j] / sim->a_ii; }
            }
            if (sim->ens || !r1_fused(sim, t)) {
                e = launch_combine(n3, sim->q, t, sim->R1, nullptr, st);
                if (e == cudaSuccess)
                    e = sim->ens ? launch_ens_condense(*sim->ens, sim->R1, sim->Z, sim->gvec, st)
                                 : launch_condense(sim->g, sim->ops, sim->R1, sim->phiB, sim->tau, sim->Z,
                                                   sim->gvec, st, 0.0);
            } else {   // the FP32-pair Schur condensation forms R1 as it reads it
                const R1Source src{sim->q, t};
                e = launch_condense(sim->g, sim->ops, sim->R1, sim->phiB, sim->tau, sim->Z, sim->gvec, st, 0.0, &src);
            }
            if (e == cudaSuccess) {
                if (sim->cfg.precision == HDGDG_MIXED)
                    e = solve_enqueue_graph<float>(sim, sim->gvec, sim->lam, i, st, sg, branch);
                else e = solve_enqueue_graph<double>(sim, sim->gvec, sim->lam, i, st, sg, branch);
            }
            if (branch && e == cudaSuccess) {
                e = cudaEventRecord(sim->fork_ev[i], st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(sim->side_stream, sim->fork_ev[i], 0);
                if (e == cudaSuccess)
                    e = launch_hist_store_dev(sim->plan.nt, sim->xt, sim->gvec, sim->w, sim->dhist + i,
                                              sim->side_stream);
                if (e == cudaSuccess) e = cudaEventRecord(sim->join_ev[i], sim->side_stream);
                if (e == cudaSuccess) pending = i;
            }
            if (e == cudaSuccess)
                e = sim->ens ? launch_ens_recover(*sim->ens, sim->Z, sim->R1, sim->lam, 1.0, sim->Qs,
                                                  sim->Ls[i], st)
                             : launch_recover(sim->g, sim->ops, sim->Z, sim->R1, sim->tau, sim->lam, beta_of(sim),
                                              1.0, sim->Qs, sim->Ls[i], st, sim->Qs32);
            Qi = sim->Qs;
        }
        if (fuse_final && i == sim->s - 1) {
            const FinalSource fin{sim->q, tf, slot, sim->q_new, sim->flags};
            if (e == cudaSuccess) e = cudaMemsetAsync(sim->flags, 0, sizeof(unsigned), st);
            if (e == cudaSuccess) e = dg_nl_enqueue(sim, Qi, Qi == sim->Qs, sim->NLs[i], st, 0.0, &fin);
        } else if (!sim->cfg.linear_only && e == cudaSuccess) {
            e = dg_nl_enqueue(sim, Qi, Qi == sim->Qs, sim->NLs[i], st, 0.0);
        }
    }
    if (pending >= 0 && e == cudaSuccess) e = cudaStreamWaitEvent(st, sim->join_ev[pending], 0);
    if (!fuse_final) {
        if (e == cudaSuccess) e = cudaMemsetAsync(sim->flags, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = launch_combine(n3, sim->q, tf, sim->q_new, sim->flags, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sim->hbuf, sim->flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sim->hbuf + 4, sim->sstats, sizeof(StepStats), cudaMemcpyDeviceToHost, st);
    return e;
}

// The captured step depends on the state buffers only: the guess history is read through the
// device table (DevHist) that one_step_graph writes before each replay.
std::vector<const void*> step_key(const hdgdg_sim* sim) { return {sim->q, sim->q_new}; }

// Each implicit stage's history table for the next replay: the host's rotated pointers, the
// number of usable solutions and the slot the step writes.
cudaError_t upload_history(hdgdg_sim* sim, cudaStream_t st) {
    const int order = guess_order(&sim->cfg);
    for (int i = 0; i < sim->s; ++i) {
        DevHist& h = sim->hhist[i];
        h = DevHist{};
        if (sim->At[i][i] == 0.0 || order <= 0) continue;
        for (int j = 0; j < order; ++j) {
            h.x[j] = sim->xhist[i][j];
            h.y[j] = sim->yhist[i][j];
        }
        h.xw = sim->xhist[i][order - 1];
        h.yw = sim->yhist[i][order - 1];
        h.avail = std::min(order, sim->n_hist[i]);
        h.has_history = h.avail > 0 ? 1 : 0;
    }
    return cudaMemcpyAsync(sim->dhist, sim->hhist, sim->s * sizeof(DevHist), cudaMemcpyHostToDevice, st);
}

void drop_step_graphs(hdgdg_sim* sim) {
    for (auto& sg : sim->step_graphs)
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
    sim->step_graphs.clear();
}

// Whole-step graphs serve implicit schemes whose boundary data do not depend on time, with the
// kernel-class timers off (their event records cannot sit inside a conditional node's body).
bool use_step_graph(const hdgdg_sim* sim) {
    if (sim->ens) return true;   // an ensemble's steps are always replayed graphs
    return !sim->cfg.host_steps && !sim->timing && !explicit_scheme(&sim->cfg) && !sim->g.dirichlet &&
           sim->body_stream != nullptr;
}

hdgdg_status one_step_graph(hdgdg_sim* sim) {
    NvtxRange nv("time_step_graph");
    cudaStream_t st = sim->stream;
    const std::vector<const void*> key = step_key(sim);
    StepGraph* sg = nullptr;
    for (auto& c : sim->step_graphs)
        if (c.key == key) sg = &c;
    if (!sg) {
        if (sim->step_graphs.size() >= 24) drop_step_graphs(sim);   // bounded cache
        StepGraph fresh;
        fresh.key = key;
        const long long l0 = launches_total();
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = step_enqueue_graph(sim, st, fresh);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
        fresh.launches = launches_total() - l0;
        count_launches((int)-fresh.launches);   // counted again at every replay
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(sim, HDGDG_ECUDA, "capturing the time step failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        const cudaError_t e3 = cudaGraphInstantiate(&fresh.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return fail(sim, HDGDG_ECUDA, "time-step graph: %s", cudaGetErrorString(e3));
        sim->step_graphs.push_back(std::move(fresh));
        sg = &sim->step_graphs.back();
    }
    CU(upload_history(sim, st));
    CU(cudaGraphLaunch(sg->exec, st));
    CU(cudaStreamSynchronize(st));
    unsigned flag[4];
    StepStats ss;
    std::memcpy(flag, sim->hbuf, sizeof(flag));
    std::memcpy(&ss, sim->hbuf + 4, sizeof(ss));
    count_launches((int)(sg->launches + (long long)(ss.cycles - sg->bodies) * sg->per_cycle));
    sim->stats.krylov_iterations += ss.its;
    sim->stats.last_krylov_iterations = ss.last_its;
    sim->stats.last_rel_residual = ss.last_rel;
    sim->stats.last_guess_order = ss.last_guess;
    const bool bad = flag[0] || flag[2] || flag[3] || ss.nonfinite || ss.notconv;
    if (bad) {   // the history slots may hold this step's partial solves: start the next solves afresh
        for (int i = 0; i < sim->s; ++i) sim->n_hist[i] = 0;
        if (flag[2]) return fail(sim, HDGDG_ECUDA, "a bounded wait of a local kernel ran out (%u)", flag[2]);
        if (flag[3]) return fail(sim, HDGDG_ECUDA, "a bounded wait of the pipelined SpMV ran out (%u)", flag[3]);
        if (ss.nonfinite) return fail(sim, HDGDG_ENONFINITE, "non-finite trace right-hand side or GMRES residual");
        if (ss.notconv) {
            sim->stats.last_krylov_iterations = ss.notconv_its;
            sim->stats.last_rel_residual = ss.notconv_rel;
            return fail(sim, HDGDG_ENOTCONVERGED, "GMRES: relative residual %.3e above the tolerance after %d iterations",
                        ss.notconv_rel, ss.notconv_its);
        }
        return fail(sim, HDGDG_ENONFINITE, "step %lld produced a non-finite state", sim->stats.steps + 1);
    }
    const int order = guess_order(&sim->cfg);
    for (int i = 0; i < sim->s && order > 0; ++i) {   // the slot written last becomes the newest
        if (sim->At[i][i] == 0.0) continue;
        double* ox = sim->xhist[i][order - 1];
        double* oy = sim->yhist[i][order - 1];
        for (int j = order - 1; j > 0; --j) {
            sim->xhist[i][j] = sim->xhist[i][j - 1];
            sim->yhist[i][j] = sim->yhist[i][j - 1];
        }
        sim->xhist[i][0] = ox;
        sim->yhist[i][0] = oy;
        sim->n_hist[i] = std::min(sim->n_hist[i] + 1, order);
    }
    std::swap(sim->q, sim->q_new);
    sim->stats.steps += 1;
    sim->t += sim->cfg.dt;
    return HDGDG_OK;
}

// Explicit SSP Runge-Kutta on the whole DG residual (the paper's RK2 DG / RK3 DG), with the
// stage increments K_i = dt M^{-1} R(q_i):
//   RK2 (Heun):        q1 = q + K1;                 q' = q + K1/2 + K2/2
//   RK3 (Shu-Osher):   q1 = q + K1;  q2 = q + K1/4 + K2/4;  q' = q + K1/6 + K2/6 + 2 K3/3
hdgdg_status explicit_step(hdgdg_sim* sim) {
    NvtxRange nv("time_step");
    const size_t n3 = 3 * sim->plan.n;
    cudaStream_t st = sim->stream;
    const double dt = sim->cfg.dt;
    auto rhs = [&](const double* qi, double* K, double ti) -> hdgdg_status {
        TimedGroup tg(sim, HDGDG_KT_DG);
        CU(launch_dg_full(sim->g, qi, sim->phiB, dt, sim->fface, K, st, ti));
        return HDGDG_OK;
    };
    const double t0 = sim->t;
    auto comb = [&](double* out, std::initializer_list<std::pair<double*, double>> terms, unsigned* flag) -> hdgdg_status {
        CombineTerms t{};
        for (auto& pr : terms) { t.X[t.n] = pr.first; t.c[t.n++] = pr.second; }
        TimedGroup tg(sim, HDGDG_KT_COMBINE);
        CU(launch_combine(n3, sim->q, t, out, flag, st));
        return HDGDG_OK;
    };
    double *K1 = sim->NLs[0], *K2 = sim->NLs[1], *K3 = sim->NLs[2];
    TRY(rhs(sim->q, K1, t0));
    TRY(comb(sim->Qs, {{K1, 1.0}}, nullptr));
    TRY(rhs(sim->Qs, K2, t0 + dt));
    CU(cudaMemsetAsync(sim->flags, 0, sizeof(unsigned), st));
    if (sim->cfg.scheme == HDGDG_RK2) {
        TRY(comb(sim->q_new, {{K1, 0.5}, {K2, 0.5}}, sim->flags));
    } else {
        TRY(comb(sim->R1, {{K1, 0.25}, {K2, 0.25}}, nullptr));
        TRY(rhs(sim->R1, K3, t0 + 0.5 * dt));
        TRY(comb(sim->q_new, {{K1, 1.0 / 6.0}, {K2, 1.0 / 6.0}, {K3, 2.0 / 3.0}}, sim->flags));
    }
    unsigned flag = 0;
    CU(cudaMemcpyAsync(&sim->hbuf[0], sim->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TRY(sync(sim));
    std::memcpy(&flag, &sim->hbuf[0], sizeof(unsigned));
    if (flag) return fail(sim, HDGDG_ENONFINITE, "step %lld produced a non-finite state", sim->stats.steps + 1);
    std::swap(sim->q, sim->q_new);
    sim->stats.steps += 1;
    sim->t += dt;
    return HDGDG_OK;
}

hdgdg_status one_step(hdgdg_sim* sim) {
    if (use_step_graph(sim)) return one_step_graph(sim);
    NvtxRange nv("time_step");
    if (explicit_scheme(&sim->cfg)) return explicit_step(sim);
    const size_t n3 = 3 * sim->plan.n;
    cudaStream_t st = sim->stream;
    for (int i = 0; i < sim->s; ++i) {
        const double* Qi = sim->q;
        double ci = 0.0;   // stage abscissa c_i = sum_j a_ij (equal for both tableaux of ARS)
        for (int j = 0; j < i; ++j) ci += sim->A[i][j];
        const double ti = sim->t + ci * sim->cfg.dt;
        if (sim->At[i][i] != 0.0) {
            CombineTerms t{};
            for (int j = 0; j < i; ++j) {
                if (sim->A[i][j] != 0.0 && !sim->cfg.linear_only) { t.X[t.n] = sim->NLs[j]; t.c[t.n++] = sim->A[i][j]; }
                if (sim->At[i][j] != 0.0) { t.X[t.n] = sim->Ls[j]; t.c[t.n++] = sim->At[i][j] / sim->a_ii; }
            }
            // the FP32-pair Schur condensation forms R1 itself, as in the step graph
            const bool fused = r1_fused(sim, t);
            if (!fused) {
                TimedGroup tg(sim, HDGDG_KT_COMBINE);
                CU(launch_combine(n3, sim->q, t, sim->R1, nullptr, st));
            }
            const R1Source src{sim->q, t};
            int its = 0;
            TRY(stage_solve_dev(sim, sim->R1, sim->Qs, sim->Ls[i], &its, ti, i, sim->Qs32, fused ? &src : nullptr));
            Qi = sim->Qs;
        }
        if (!sim->cfg.linear_only) {
            TimedGroup tg(sim, HDGDG_KT_DG);
            CU(dg_nl_enqueue(sim, Qi, Qi == sim->Qs, sim->NLs[i], st, ti));
        }
    }
    CombineTerms t{};
    for (int i = 0; i < sim->s; ++i) {
        if (sim->b[i] != 0.0 && !sim->cfg.linear_only) { t.X[t.n] = sim->NLs[i]; t.c[t.n++] = sim->b[i]; }
        if (sim->bt[i] != 0.0) { t.X[t.n] = sim->Ls[i]; t.c[t.n++] = sim->bt[i] / sim->a_ii; }
    }
    CU(cudaMemsetAsync(sim->flags, 0, sizeof(unsigned), st));
    {
        TimedGroup tg(sim, HDGDG_KT_COMBINE);
        CU(launch_combine(n3, sim->q, t, sim->q_new, sim->flags, st));
    }
    unsigned flag[4] = {0, 0, 0, 0};   // non-finite, (setup), tensor-core wait, SpMV wait ran out
    CU(cudaMemcpyAsync(&sim->hbuf[0], sim->flags, sizeof(flag), cudaMemcpyDeviceToHost, st));
    TRY(sync(sim));
    std::memcpy(flag, &sim->hbuf[0], sizeof(flag));
    if (flag[2]) return fail(sim, HDGDG_ECUDA, "a bounded wait of a local kernel ran out (%u)", flag[2]);
    if (flag[3]) return fail(sim, HDGDG_ECUDA, "a bounded wait of the pipelined SpMV ran out (%u)", flag[3]);
    if (flag[0]) return fail(sim, HDGDG_ENONFINITE, "step %lld produced a non-finite state", sim->stats.steps + 1);
    std::swap(sim->q, sim->q_new);
    sim->stats.steps += 1;
    sim->t += sim->cfg.dt;
    return HDGDG_OK;
}

hdgdg_status setup(hdgdg_sim* sim, const double* bottom_b) {
    const hdgdg_config* c = &sim->cfg;
    const Plan& p = sim->plan;
    const Geom& g = sim->g;
    const int P = g.P, Np = g.Np;
    // phi_B = g (H0 - b) at the nodes; tau = max of sqrt(phi_B) over both sides of each edge node
    std::vector<double> phiB(p.n), tau((size_t)g.n_edges * P);
    for (size_t k = 0; k < p.n; ++k) {
        const double b = bottom_b ? bottom_b[k] : 0.0;
        phiB[k] = c->g * (c->H0 - b);
        if (!std::isfinite(phiB[k])) return fail(sim, HDGDG_ENONFINITE, "non-finite bottom at node %zu", k);
        if (!(phiB[k] > 0.0))
            return fail(sim, HDGDG_EINVAL, "reference depth H0 - b must be positive (node %zu)", k);
    }
    for (int r = 0; r < g.n_edges; ++r) {
        int em, fm, ep, fp;
        edge_sides(r, g, &em, &fm, &ep, &fp);
        for (int b = 0; b < P; ++b) {
            // a wall edge has one side: tau = sqrt(phi_B) of that side
            const double a1 = em >= 0 ? std::sqrt(phiB[(size_t)em * Np + face_node(fm, b, P)]) : 0.0;
            const double a2 = ep >= 0 ? std::sqrt(phiB[(size_t)ep * Np + face_node(fp, b, P)]) : 0.0;
            tau[(size_t)r * P + b] = a1 > a2 ? a1 : a2;
        }
    }
    TRY(dalloc(sim, &sim->phiB, p.n));
    TRY(dalloc(sim, &sim->tau, tau.size()));
    if (c->dt_per_instance) {   // per-instance time steps as factors of cfg.dt
        std::vector<double> f(g.batch);
        for (int i = 0; i < g.batch; ++i) {
            f[i] = c->dt_per_instance[i] / c->dt;
            sim->dt_fingerprint += (i + 1) * c->dt_per_instance[i];
            if (!std::isfinite(f[i]) || !(f[i] > 0.0))
                return fail(sim, HDGDG_EINVAL, "time step of instance %d is not positive", i);
        }
        double* d = nullptr;
        TRY(dalloc(sim, &d, g.batch));
        CU(cudaMemcpy(d, f.data(), g.batch * sizeof(double), cudaMemcpyHostToDevice));
        sim->g.dt_scale = d;
    }
    if (explicit_scheme(c)) {
        for (double** v : {&sim->q, &sim->q_new, &sim->R1, &sim->Qs}) TRY(dalloc(sim, v, 3 * p.n));
        for (int i = 0; i < 3; ++i) TRY(dalloc(sim, &sim->NLs[i], 3 * p.n));
        TRY(dalloc(sim, &sim->fface, p.nt));
        TRY(dalloc(sim, &sim->red, reduction_scratch_doubles(p.m, g.n_edges, g.P)));
    CU(cudaMemset(sim->red, 0, sizeof(double)));   // the reductions' ticket counter starts at zero
        TRY(dalloc(sim, &sim->mred, mass_scratch_doubles()));
        TRY(dalloc(sim, &sim->dvals, 4 * (size_t)(p.m + 2) + 16));
        TRY(dalloc(sim, &sim->flags, 16));
        CU(cudaMallocHost(&sim->hbuf, (4 * (size_t)(p.m + 2) + 16) * sizeof(double)));
        CU(cudaMemcpyAsync(sim->phiB, phiB.data(), p.n * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
        CU(cudaMemcpyAsync(sim->tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
        CU(cudaStreamSynchronize(sim->stream));
        return HDGDG_OK;
    }
    TRY(dalloc(sim, &sim->Ainv, (size_t)g.n_el * p.NV * p.NV));
    TRY(dalloc(sim, &sim->Stil, (size_t)g.n_edges * 6 * p.NF * p.NF));
    TRY(dalloc(sim, &sim->Scol, (size_t)g.n_edges * 6));
    TRY(dalloc(sim, &sim->Minv, (size_t)g.n_edges * p.NF * p.NF));
    TRY(dalloc(sim, &sim->Srr, (size_t)g.n_edges * p.NF * p.NF));
    for (double** v : {&sim->q, &sim->q_new, &sim->R1, &sim->Z, &sim->Qs}) TRY(dalloc(sim, v, 3 * p.n));
    for (int i = 0; i < p.s; ++i) {
        TRY(dalloc(sim, &sim->NLs[i], 3 * p.n));
        TRY(dalloc(sim, &sim->Ls[i], 3 * p.n));
    }
    for (double** v : {&sim->gvec, &sim->xt, &sim->lam, &sim->w, &sim->fface}) TRY(dalloc(sim, v, p.nt));
    for (int i = 0; i < p.s; ++i)
        for (int h = 0; h < guess_order(c); ++h) {
            TRY(dalloc(sim, &sim->xhist[i][h], p.nt));
            TRY(dalloc(sim, &sim->yhist[i][h], p.nt));
        }
    if (c->precision == HDGDG_MIXED) {
        if (!matrix_free(c)) {
            TRY(dalloc(sim, &sim->Stil32, (size_t)g.n_edges * 6 * p.NF * p.NF));
            if (c->residual_f32x2) TRY(dalloc(sim, &sim->Stil_lo, (size_t)g.n_edges * 6 * p.NF * p.NF));
        }
        TRY(dalloc(sim, &sim->V32, (size_t)(p.m + 1) * p.nt));
        TRY(dalloc(sim, &sim->w32, (matrix_free(c) ? 3 : 1) * p.nt));   // matrix-free: w1 and two alternating outputs
    } else {
        TRY(dalloc(sim, &sim->V, (size_t)(p.m + 1) * p.nt));
    }
    TRY(dalloc(sim, &sim->red, reduction_scratch_doubles(p.m, g.n_edges, g.P)));
    CU(cudaMemset(sim->red, 0, sizeof(double)));   // the reductions' ticket counter starts at zero
    TRY(dalloc(sim, &sim->mred, mass_scratch_doubles()));
    TRY(dalloc(sim, &sim->dvals, 4 * (size_t)(p.m + 2) + 16));
    TRY(dalloc(sim, &sim->flags, 16));
    TRY(dalloc(sim, &sim->ctl, 1));
    TRY(dalloc(sim, &sim->sctl, 1));
    TRY(dalloc(sim, &sim->sstats, 1));
    TRY(dalloc(sim, &sim->dhist, kMaxStages));
    CU(cudaMallocHost(&sim->hhist, kMaxStages * sizeof(DevHist)));
    TRY(dalloc(sim, &sim->dls, kLsSlots));
    if (!c->host_steps) {
        CU(cudaStreamCreateWithFlags(&sim->body_stream, cudaStreamNonBlocking));
        CU(cudaStreamCreateWithFlags(&sim->side_stream, cudaStreamNonBlocking));
        for (int i = 0; i < kMaxStages; ++i) {
            CU(cudaEventCreateWithFlags(&sim->fork_ev[i], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&sim->join_ev[i], cudaEventDisableTiming));
        }
    }
    CU(cudaMallocHost(&sim->hbuf, (4 * (size_t)(p.m + 2) + 16) * sizeof(double)));
    for (int i = 0; i < p.s; ++i) {
        CU(cudaMemsetAsync(sim->NLs[i], 0, 3 * p.n * sizeof(double), sim->stream));
        CU(cudaMemsetAsync(sim->Ls[i], 0, 3 * p.n * sizeof(double), sim->stream));
    }
    CU(cudaMemcpyAsync(sim->phiB, phiB.data(), p.n * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
    CU(cudaMemcpyAsync(sim->tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
    // setup-only temporaries: element Schur blocks and the full 7-block rows
    double *Se = nullptr, *S7 = nullptr;
    CU(cudaMalloc(&Se, (size_t)g.n_el * p.NT * p.NT * sizeof(double)));
    cudaError_t e2 = cudaMalloc(&S7, (size_t)g.n_edges * 7 * p.NF * p.NF * sizeof(double));
    if (e2 != cudaSuccess) {
        cudaFree(Se);
        cudaGetLastError();
        return fail(sim, HDGDG_ENOMEM, "setup temporaries: %s", cudaGetErrorString(e2));
    }
    int* dsing = reinterpret_cast<int*>(sim->flags) + 1;
    CU(cudaMemsetAsync(dsing, 0, sizeof(int), sim->stream));
    cudaError_t e = launch_build_local(g, sim->phiB, sim->tau, c->dt * sim->a_ii, sim->Ainv, Se, dsing, sim->stream);
    if (e == cudaSuccess)
        e = launch_assemble_trace(g, Se, S7, sim->Srr, sim->Minv, sim->Stil, sim->Scol, dsing, sim->stream);
    if (e == cudaSuccess && c->precision == HDGDG_MIXED && matrix_free(c)) {
        sim->Minv16 = nullptr;   // (allocated below, after the setup temporaries are released)
    } else if (e == cudaSuccess && c->precision == HDGDG_MIXED) {
        if (sim->Stil_lo) {   // hi part = the FP32 copy of the inner cycles, lo part = the rest
            e = launch_split_f32x2(sim->Stil, sim->Stil32, sim->Stil_lo, (size_t)g.n_edges * 6 * p.NF * p.NF,
                                   sim->stream);
            // M^{-1} (no longer needed in FP64 once S~ exists) as FP32 pairs for the back-transformation
            if (e == cudaSuccess) e = launch_split_pairs_inplace(sim->Minv, (size_t)g.n_edges * p.NF * p.NF, sim->stream);
            sim->minv_pairs = e == cudaSuccess;
        }
        else
            e = launch_to_f32(sim->Stil, sim->Stil32, (size_t)g.n_edges * 6 * p.NF * p.NF, sim->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    cudaFree(Se);
    cudaFree(S7);
    if (e != cudaSuccess) return fail(sim, HDGDG_ECUDA, "operator setup failed: %s", cudaGetErrorString(e));
    int sing = 0;
    CU(cudaMemcpy(&sing, dsing, sizeof(int), cudaMemcpyDeviceToHost));
    if (sing) return fail(sim, HDGDG_EINVAL, "a local operator block is singular");
    sim->ops.kind = 0;
    sim->ops.Ainv = sim->Ainv;
    if (local_schur(c)) {
        const bool x2 = c->local_precision == HDGDG_LOCAL_F32X2;
        TRY(dalloc(sim, &sim->Sphi, (size_t)g.n_el * Np * Np));
        TRY(dalloc(sim, &sim->Saux, 4 * (size_t)g.n_el * Np));
        TRY(dalloc(sim, &sim->Seg, 2 * (size_t)g.batch * Np));
        CU(launch_schur_setup(g, sim->Ainv, sim->phiB, sim->tau, c->dt * sim->a_ii, x2, sim->Sphi, sim->Saux,
                              sim->Seg, sim->stream));
        sim->ops.kind = x2 ? 3 : 0;
        sim->ops.schur = true;
        sim->ops.error = reinterpret_cast<int*>(sim->flags) + 2;   // the staged tile's bounded waits
        if (c->precision == HDGDG_MIXED && c->dg_precision == 0 && !explicit_scheme(c)) {
            // the DG residual's FP32 copies and the recovery's FP32 stage values (the same roundings
            // the FP32 residual took from the FP64 values)
            TRY(dalloc(sim, &sim->Qs32, 3 * p.n));
            TRY(dalloc(sim, &sim->phiB32, p.n));
            TRY(dalloc(sim, &sim->tau32, (size_t)g.n_edges * g.P));
            CU(launch_to_f32(sim->phiB, sim->phiB32, p.n, sim->stream));
            CU(launch_to_f32(sim->tau, sim->tau32, (size_t)g.n_edges * g.P, sim->stream));
        }
        sim->ops.S = sim->Sphi;
        sim->ops.aux = sim->Saux;
        sim->ops.EG = sim->Seg;
        if (matrix_free(c)) {   // FP32 copies (the pairs' high parts) for the inner cycles, FP32 M^{-1}
            const size_t nS = (size_t)g.n_el * Np * Np, nA = 4 * (size_t)g.n_el * Np, nE = 2 * (size_t)g.batch * Np;
            float *S32 = nullptr, *aux32 = nullptr, *EG32 = nullptr;
            double *ybuf = nullptr, *hm = nullptr, *hp = nullptr;
            TRY(dalloc(sim, &S32, nS));
            TRY(dalloc(sim, &aux32, nA));
            TRY(dalloc(sim, &EG32, nE));
            TRY(dalloc(sim, &sim->Minv16, (size_t)g.n_edges * p.NF * p.NF));
            TRY(dalloc(sim, &sim->Mscale, (size_t)g.n_edges));
            TRY(dalloc(sim, &ybuf, p.nt));
            if (!sim->tau32) {
                TRY(dalloc(sim, &sim->tau32, (size_t)g.n_edges * g.P));
                CU(launch_to_f32(sim->tau, sim->tau32, (size_t)g.n_edges * g.P, sim->stream));
            }
            sim->mf.tau32 = sim->tau32;
            double* tau2 = nullptr;   // FP32 pairs in place of a copy of tau
            TRY(dalloc(sim, &tau2, (size_t)g.n_edges * g.P));
            CU(cudaMemcpyAsync(tau2, sim->tau, (size_t)g.n_edges * g.P * sizeof(double), cudaMemcpyDeviceToDevice,
                               sim->stream));
            CU(launch_split_pairs_inplace(tau2, (size_t)g.n_edges * g.P, sim->stream));
            sim->mf.tau2 = tau2;
            TRY(dalloc(sim, &hm, p.nt));
            TRY(dalloc(sim, &hp, p.nt));
            CU(launch_pair_hi(sim->Sphi, S32, nS, sim->stream));
            CU(launch_pair_hi(sim->Saux, aux32, nA, sim->stream));
            CU(launch_pair_hi(sim->Seg, EG32, nE, sim->stream));
            CU(launch_precond_f16(sim->Minv, g.n_edges, p.NF, sim->Minv16, sim->Mscale, sim->stream));
            sim->mf.S32 = S32;
            sim->mf.aux32 = aux32;
            sim->mf.EG32 = EG32;
            sim->mf.S2 = sim->Sphi;
            sim->mf.aux2 = sim->Saux;
            sim->mf.EG2 = sim->Seg;
            sim->mf.Minv.h = sim->Minv16;
            sim->mf.Minv.scale = sim->Mscale;
            sim->mf.tau = sim->tau;
            sim->mf.ybuf = ybuf;
            sim->mf.hm = hm;
            sim->mf.hp = hp;
        }
        if (g.n_el >= 4096) {   // pick the tiles on this handle's operators, then clear the scratch
            CU(launch_autotune_local(g, sim->ops, sim->R1, sim->Z, sim->tau, sim->lam, sim->Qs, sim->NLs[0],
                                     sim->stream));
            if (matrix_free(c)) {
                CU(cudaMemsetAsync(sim->V32, 0, p.nt * sizeof(float), sim->stream));
                CU(cudaMemsetAsync(sim->xt, 0, p.nt * sizeof(double), sim->stream));
                CU(cudaMemsetAsync(sim->gvec, 0, p.nt * sizeof(double), sim->stream));
                CU(launch_mf_autotune(g, sim->mf, sim->V32, sim->w32, sim->xt, sim->gvec, sim->w, beta_of(sim),
                                      sim->stream, &sim->trace_tile, &sim->trace_prefetch));
            }
            for (double* v : {sim->R1, sim->Z, sim->Qs, sim->NLs[0]})
                CU(cudaMemsetAsync(v, 0, 3 * p.n * sizeof(double), sim->stream));
            CU(cudaMemsetAsync(sim->lam, 0, p.nt * sizeof(double), sim->stream));
        }
    } else if (c->local_precision == HDGDG_LOCAL_FP32) {
        const size_t n = (size_t)g.n_el * p.NV * p.NV;
        TRY(dalloc(sim, &sim->Ainv32, n));
        CU(launch_to_f32(sim->Ainv, sim->Ainv32, n, sim->stream));
        sim->ops.kind = 1;
        sim->ops.Ainv32 = sim->Ainv32;
    } else if (c->local_precision == HDGDG_LOCAL_F32X2) {
        const size_t n = (size_t)g.n_el * p.NV * p.NV;
        TRY(dalloc(sim, &sim->Ahi, n));
        TRY(dalloc(sim, &sim->Alo, n));
        CU(launch_split_f32x2(sim->Ainv, sim->Ahi, sim->Alo, n, sim->stream));
        sim->ops.kind = 3;
        sim->ops.Ahi = sim->Ahi;
        sim->ops.Alo = sim->Alo;
        if (g.n_el >= 4096) {   // pick the kernels' tile on this handle's operators, then clear the scratch
            CU(launch_autotune_local(g, sim->ops, sim->R1, sim->Z, sim->tau, sim->lam, sim->Qs, sim->NLs[0],
                                     sim->stream));
            for (double* v : {sim->R1, sim->Z, sim->Qs, sim->NLs[0]})
                CU(cudaMemsetAsync(v, 0, 3 * p.n * sizeof(double), sim->stream));
            CU(cudaMemsetAsync(sim->lam, 0, p.nt * sizeof(double), sim->stream));
        }
    } else if (c->local_precision == HDGDG_LOCAL_BF16 || c->local_precision == HDGDG_LOCAL_BF16_SPLIT) {
        // one operator for every element: phi_B constant and one time step
        for (size_t k = 1; k < p.n; ++k)
            if (phiB[k] != phiB[0])
                return fail(sim, HDGDG_EINVAL, "tensor-core local contractions need a flat bottom");
        if (c->dt_per_instance)
            for (int i = 0; i < g.batch; ++i)
                if (c->dt_per_instance[i] != c->dt)
                    return fail(sim, HDGDG_EINVAL, "tensor-core local contractions need one time step");
        const bool split = c->local_precision == HDGDG_LOCAL_BF16_SPLIT;
        uint8_t* img = nullptr;
        TRY(dalloc(sim, &img, split ? tc_split_image_bytes(P) : tc_image_bytes(P)));
        sim->tc_image = img;
        if (split) CU(launch_tc_split_image(g, sim->Ainv, img, sim->stream));
        else CU(launch_tc_image(g, sim->Ainv, img, sim->stream));
        sim->ops.kind = split ? 4 : 2;
        sim->ops.image = img;
        sim->ops.error = reinterpret_cast<int*>(sim->flags) + 2;
    }
    CU(cudaMemsetAsync(sim->flags, 0, 16, sim->stream));
    CU(cudaStreamSynchronize(sim->stream));
    return HDGDG_OK;
}

hdgdg_status upload3(hdgdg_sim* sim, double* dst, const double* src, size_t count) {
    CU(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
    return HDGDG_OK;
}

// The device's address of a pinned host buffer (page-locked, mapped: the GPU reads and writes it
// directly over the host link), or nullptr for other host memory.
const void* device_view(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// User (h, hu, hv) on the host -> state q = (phi_eta, U, V) in dst; *ok false when a value is
// not finite or the depth is not positive.  Pinned host buffers are read by the conversion kernel
// itself; other host memory is first copied to the device.
hdgdg_status load_user_state(hdgdg_sim* sim, const double* h, const double* hu, const double* hv, double* dst,
                             bool* ok) {
    const size_t n = sim->plan.n;
    const double* dh = static_cast<const double*>(device_view(h));
    const double* dhu = static_cast<const double*>(device_view(hu));
    const double* dhv = static_cast<const double*>(device_view(hv));
    if (!dh || !dhu || !dhv) {
        double* stg = sim->NLs[0];
        TRY(upload3(sim, stg, h, n));
        TRY(upload3(sim, stg + n, hu, n));
        TRY(upload3(sim, stg + 2 * n, hv, n));
        dh = stg;
        dhu = stg + n;
        dhv = stg + 2 * n;
    }
    CU(cudaMemsetAsync(sim->flags, 0, sizeof(unsigned), sim->stream));
    CU(launch_user_to_state(sim->g, dh, dhu, dhv, sim->phiB, sim->cfg.g, dst, sim->flags, sim->stream));
    CU(cudaMemcpyAsync(sim->hbuf, sim->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, sim->stream));
    TRY(sync(sim));
    unsigned bad = 0;
    std::memcpy(&bad, sim->hbuf, sizeof(unsigned));
    *ok = bad == 0;
    return HDGDG_OK;
}

hdgdg_status download(hdgdg_sim* sim, double* dst, const double* src, size_t count) {
    CU(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    return sync(sim);
}

}  // namespace

extern "C" {

size_t hdgdg_bytes_required(const hdgdg_config* cfg) {
    if (!valid(cfg)) return 0;
    const Plan p = make_plan(cfg);
    return p.persistent + p.setup_temp;
}

hdgdg_status hdgdg_node_coords(const hdgdg_config* cfg, double* x, double* y) {
    if (!valid(cfg) || !x || !y) return HDGDG_EINVAL;
    double xi[kMaxP];
    Geom g = make_geom(cfg, xi);
    for (int e = 0; e < g.n_el_inst; ++e) {
        const int ex = e % g.N, ey = e / g.N;
        for (int j = 0; j < g.P; ++j)
            for (int i = 0; i < g.P; ++i) {
                x[(size_t)e * g.Np + j * g.P + i] = g.x0 + (ex + (1.0 + xi[i]) / 2.0) * g.h;
                y[(size_t)e * g.Np + j * g.P + i] = g.x0 + (ey + (1.0 + xi[j]) / 2.0) * g.h;
            }
    }
    return HDGDG_OK;
}

hdgdg_status hdgdg_gll(int degree_k, double* nodes, double* weights) {
    if (degree_k < 1 || degree_k > kMaxP - 1 || !nodes || !weights) return HDGDG_EINVAL;
    double D[kMaxP * kMaxP];
    gll_tables(degree_k, nodes, weights, D);
    return HDGDG_OK;
}

const char* hdgdg_last_error(const hdgdg_sim* sim) {
    if (!sim) return "no handle";
    return sim->err.c_str();
}

void hdgdg_destroy(hdgdg_sim* sim) {
    if (!sim) return;
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    flush_timers(sim);
    for (auto& cg : sim->cycle_graph) drop_graph(sim, cg);
    drop_step_graphs(sim);
    if (sim->body_stream) cudaStreamDestroy(sim->body_stream);
    if (sim->side_stream) cudaStreamDestroy(sim->side_stream);
    for (int i = 0; i < kMaxStages; ++i) {
        if (sim->fork_ev[i]) cudaEventDestroy(sim->fork_ev[i]);
        if (sim->join_ev[i]) cudaEventDestroy(sim->join_ev[i]);
    }
    for (cudaEvent_t e : sim->ev_pool) cudaEventDestroy(e);
    for (void* p : sim->allocs) cudaFree(p);
    if (sim->hbuf) cudaFreeHost(sim->hbuf);
    if (sim->hhist) cudaFreeHost(sim->hhist);
    if (sim->own_stream && sim->stream) cudaStreamDestroy(sim->stream);
    delete sim;
}

hdgdg_status hdgdg_create(const hdgdg_config* cfg, const double* bottom_b, void* cuda_stream,
                          hdgdg_sim** out) {
    if (!out) return HDGDG_EINVAL;
    *out = nullptr;
    if (!valid(cfg)) return HDGDG_EINVAL;
    hdgdg_sim* sim = new (std::nothrow) hdgdg_sim();
    if (!sim) return HDGDG_ENOMEM;
    sim->cfg = *cfg;
    sim->plan = make_plan(cfg);
    sim->g = make_geom(cfg, nullptr);
    if (explicit_scheme(cfg)) {
        sim->s = 3;
        std::memset(sim->A, 0, sizeof(sim->A));
        std::memset(sim->At, 0, sizeof(sim->At));
    } else {
        scheme_tables(cfg->scheme, sim->A, sim->At, sim->b, sim->bt, &sim->s);
    }
    sim->a_ii = sim->At[1][1];
    for (int i = 0; i < sim->s; ++i) {
        if (sim->At[i][i] != 0.0 && sim->At[i][i] != sim->a_ii) {
            hdgdg_destroy(sim);
            return HDGDG_EINVAL;
        }
    }
    if (cuda_stream) {
        sim->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            hdgdg_destroy(sim);
            return HDGDG_ECUDA;
        }
        sim->own_stream = true;
    }
    hdgdg_status st = setup(sim, bottom_b);
    if (st != HDGDG_OK) {
        // keep the handle so the caller can read the message; it may only be destroyed
        *out = sim;
        return st;
    }
    *out = sim;
    return HDGDG_OK;
}

hdgdg_status hdgdg_set_state(hdgdg_sim* sim, const double* h, const double* hu, const double* hv) {
    if (!sim || !h || !hu || !hv) return fail(sim, HDGDG_EINVAL, "NULL argument to set_state");
    bool ok = false;
    TRY(load_user_state(sim, h, hu, hv, sim->q, &ok));
    if (!ok) {
        sim->have_state = false;
        return fail(sim, HDGDG_ENONFINITE, "state has a non-finite value or non-positive depth");
    }
    sim->have_state = true;
    sim->stats = hdgdg_stats{};
    sim->t = 0.0;
    for (int i = 0; i < kMaxStages; ++i) sim->n_hist[i] = 0;   // a new trajectory: no guess history
    return HDGDG_OK;
}

hdgdg_status hdgdg_update_state(hdgdg_sim* sim, const double* h, const double* hu, const double* hv) {
    if (!sim || !h || !hu || !hv) return fail(sim, HDGDG_EINVAL, "NULL argument to update_state");
    if (!sim->have_state) return fail(sim, HDGDG_ESTATE, "update_state before set_state");
    bool ok = false;
    TRY(load_user_state(sim, h, hu, hv, sim->q_new, &ok));   // q_new is free between steps
    if (!ok) return fail(sim, HDGDG_ENONFINITE, "state has a non-finite value or non-positive depth");
    std::swap(sim->q, sim->q_new);
    return HDGDG_OK;
}

hdgdg_status hdgdg_step(hdgdg_sim* sim, int n_steps) {
    if (!sim) return HDGDG_EINVAL;
    if (n_steps < 0) return fail(sim, HDGDG_EINVAL, "n_steps < 0");
    if (!sim->have_state) return fail(sim, HDGDG_ESTATE, "step before set_state");
    for (int k = 0; k < n_steps; ++k) {
        const long long l0 = launches_total();
        const hdgdg_status st = one_step(sim);
        sim->stats.kernel_launches += launches_total() - l0;
        if (st != HDGDG_OK) return st;
    }
    return HDGDG_OK;
}

hdgdg_status hdgdg_get_state(hdgdg_sim* sim, double* h, double* hu, double* hv) {
    if (!sim || !h || !hu || !hv) return fail(sim, HDGDG_EINVAL, "NULL argument to get_state");
    if (!sim->have_state) return fail(sim, HDGDG_ESTATE, "get_state before set_state");
    const size_t n = sim->plan.n;
    double* dh = static_cast<double*>(const_cast<void*>(device_view(h)));
    double* dhu = static_cast<double*>(const_cast<void*>(device_view(hu)));
    double* dhv = static_cast<double*>(const_cast<void*>(device_view(hv)));
    if (dh && dhu && dhv) {   // pinned: the conversion kernel writes the caller's buffers
        CU(launch_state_to_user(sim->g, sim->q, sim->phiB, sim->cfg.g, dh, dhu, dhv, sim->stream));
        return sync(sim);
    }
    double* stg = sim->NLs[0];
    CU(launch_state_to_user(sim->g, sim->q, sim->phiB, sim->cfg.g, stg, stg + n, stg + 2 * n, sim->stream));
    CU(cudaMemcpyAsync(h, stg, n * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    CU(cudaMemcpyAsync(hu, stg + n, n * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    CU(cudaMemcpyAsync(hv, stg + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    return sync(sim);
}

}  // extern "C"

// ---- checkpoint / resume -------------------------------------------------------------------
namespace {
struct CheckpointHeader {
    char magic[8];                 // "HDGDGCK1"
    int n_side, degree_k, scheme, precision, boundary, batch, local_precision, guess, stages;
    long long n_state, n_trace;    // doubles in the state, in one trace vector
    double dt, g, H0, x0, length;
    double dt_fingerprint;         // order-sensitive sum of the batch's per-instance time steps
    double t;
    hdgdg_stats stats;
    int n_hist[kMaxStages];        // guess history kept per stage (newest first)
};

int history_slots(const hdgdg_sim* sim) { return explicit_scheme(&sim->cfg) ? 0 : guess_order(&sim->cfg); }

size_t checkpoint_size(const hdgdg_sim* sim) {
    size_t b = sizeof(CheckpointHeader) + 3 * sim->plan.n * sizeof(double);
    for (int i = 0; i < sim->s; ++i) b += 2 * (size_t)sim->n_hist[i] * sim->plan.nt * sizeof(double);
    return b;
}

void fill_header(const hdgdg_sim* sim, CheckpointHeader* h) {
    std::memset(h, 0, sizeof(*h));
    std::memcpy(h->magic, "HDGDGCK1", 8);
    const hdgdg_config& c = sim->cfg;
    h->n_side = c.n_side;
    h->degree_k = c.degree_k;
    h->scheme = c.scheme;
    h->precision = c.precision;
    h->boundary = c.boundary;
    h->batch = sim->g.batch;
    h->local_precision = c.local_precision;
    h->guess = history_slots(sim);
    h->stages = sim->s;
    h->n_state = (long long)(3 * sim->plan.n);
    h->n_trace = (long long)sim->plan.nt;
    h->dt = c.dt;
    h->g = c.g;
    h->H0 = c.H0;
    h->x0 = c.x0;
    h->length = c.length;
    h->dt_fingerprint = sim->dt_fingerprint;
}
}  // namespace

extern "C" {

size_t hdgdg_checkpoint_bytes(hdgdg_sim* sim) {
    if (!sim || !sim->have_state) return 0;
    return checkpoint_size(sim);
}

hdgdg_status hdgdg_save_checkpoint(hdgdg_sim* sim, void* buf, size_t bytes) {
    if (!sim || !buf) return fail(sim, HDGDG_EINVAL, "NULL argument to save_checkpoint");
    if (!sim->have_state) return fail(sim, HDGDG_ESTATE, "save_checkpoint before set_state");
    if (bytes < checkpoint_size(sim))
        return fail(sim, HDGDG_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", bytes, checkpoint_size(sim));
    auto* h = static_cast<CheckpointHeader*>(buf);
    fill_header(sim, h);
    h->t = sim->t;
    h->stats = sim->stats;
    for (int i = 0; i < kMaxStages; ++i) h->n_hist[i] = i < sim->s ? sim->n_hist[i] : 0;
    char* p = static_cast<char*>(buf) + sizeof(CheckpointHeader);
    const size_t nq = 3 * sim->plan.n * sizeof(double), nt = sim->plan.nt * sizeof(double);
    CU(cudaMemcpyAsync(p, sim->q, nq, cudaMemcpyDeviceToHost, sim->stream));
    p += nq;
    for (int i = 0; i < sim->s; ++i)
        for (int j = 0; j < sim->n_hist[i]; ++j) {
            CU(cudaMemcpyAsync(p, sim->xhist[i][j], nt, cudaMemcpyDeviceToHost, sim->stream));
            CU(cudaMemcpyAsync(p + nt, sim->yhist[i][j], nt, cudaMemcpyDeviceToHost, sim->stream));
            p += 2 * nt;
        }
    return sync(sim);
}

hdgdg_status hdgdg_load_checkpoint(hdgdg_sim* sim, const void* buf, size_t bytes) {
    if (!sim || !buf) return fail(sim, HDGDG_EINVAL, "NULL argument to load_checkpoint");
    if (bytes < sizeof(CheckpointHeader)) return fail(sim, HDGDG_EINVAL, "checkpoint shorter than its header");
    const auto* h = static_cast<const CheckpointHeader*>(buf);
    CheckpointHeader mine;
    fill_header(sim, &mine);
    if (std::memcmp(h->magic, mine.magic, 8) != 0) return fail(sim, HDGDG_EINVAL, "not a checkpoint of this library");
    if (h->n_side != mine.n_side || h->degree_k != mine.degree_k || h->scheme != mine.scheme ||
        h->precision != mine.precision || h->boundary != mine.boundary || h->batch != mine.batch ||
        h->local_precision != mine.local_precision || h->guess != mine.guess || h->stages != mine.stages ||
        h->n_state != mine.n_state || h->n_trace != mine.n_trace || h->dt != mine.dt || h->g != mine.g ||
        h->H0 != mine.H0 || h->x0 != mine.x0 || h->length != mine.length ||
        h->dt_fingerprint != mine.dt_fingerprint)
        return fail(sim, HDGDG_EINVAL, "checkpoint of a different configuration");
    size_t need = sizeof(CheckpointHeader) + 3 * sim->plan.n * sizeof(double);
    for (int i = 0; i < sim->s; ++i) {
        if (h->n_hist[i] < 0 || h->n_hist[i] > mine.guess) return fail(sim, HDGDG_EINVAL, "corrupt checkpoint history");
        need += 2 * (size_t)h->n_hist[i] * sim->plan.nt * sizeof(double);
    }
    if (bytes < need) return fail(sim, HDGDG_EINVAL, "checkpoint of %zu bytes, %zu expected", bytes, need);
    const char* p = static_cast<const char*>(buf) + sizeof(CheckpointHeader);
    const size_t nq = 3 * sim->plan.n * sizeof(double), nt = sim->plan.nt * sizeof(double);
    CU(cudaMemcpyAsync(sim->q, p, nq, cudaMemcpyHostToDevice, sim->stream));
    p += nq;
    for (int i = 0; i < sim->s; ++i)
        for (int j = 0; j < h->n_hist[i]; ++j) {
            CU(cudaMemcpyAsync(sim->xhist[i][j], p, nt, cudaMemcpyHostToDevice, sim->stream));
            CU(cudaMemcpyAsync(sim->yhist[i][j], p + nt, nt, cudaMemcpyHostToDevice, sim->stream));
            p += 2 * nt;
        }
    TRY(sync(sim));
    for (int i = 0; i < kMaxStages; ++i) sim->n_hist[i] = i < sim->s ? h->n_hist[i] : 0;
    sim->t = h->t;
    sim->stats = h->stats;
    sim->have_state = true;
    return HDGDG_OK;
}

hdgdg_status hdgdg_get_stats(hdgdg_sim* sim, hdgdg_stats* out) {
    if (!sim || !out) return fail(sim, HDGDG_EINVAL, "NULL argument to get_stats");
    if (sim->have_state) {
        CU(launch_mass(sim->g, sim->q, sim->mred, dv_nrm(sim), sim->stream));
        CU(cudaMemcpyAsync(sim->hbuf, dv_nrm(sim), sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
        TRY(sync(sim));
        sim->stats.mass = sim->hbuf[0];
    }
    *out = sim->stats;
    out->time = sim->t;
    out->local_tile_condense = sim->ops.tile_condense;
    out->local_tile_recover = sim->ops.tile_recover;
    out->trace_tile = sim->trace_tile;
    out->trace_tile_prefetch = sim->trace_prefetch;
    return HDGDG_OK;
}

hdgdg_status hdgdg_eval_nl(hdgdg_sim* sim, const double* q, double* out) {
    if (!sim || !q || !out) return fail(sim, HDGDG_EINVAL, "NULL argument to eval_nl");
    const size_t n3 = 3 * sim->plan.n;
    TRY(upload3(sim, sim->R1, q, n3));
    CU(launch_dg_nl(sim->g, sim->R1, sim->phiB, sim->tau, 1.0, sim->fface, sim->Qs, sim->stream, sim->t));
    return download(sim, out, sim->Qs, n3);
}

hdgdg_status hdgdg_condense_rhs(hdgdg_sim* sim, const double* R1, double* out) {
    if (sim && explicit_scheme(&sim->cfg)) return fail(sim, HDGDG_EINVAL, "explicit scheme: no implicit stage");
    if (!sim || !R1 || !out) return fail(sim, HDGDG_EINVAL, "NULL argument to condense_rhs");
    TRY(upload3(sim, sim->R1, R1, 3 * sim->plan.n));
    CU(launch_condense(sim->g, sim->ops, sim->R1, sim->phiB, sim->tau, sim->Z, sim->gvec, sim->stream, sim->t));
    return download(sim, out, sim->gvec, sim->plan.nt);
}

hdgdg_status hdgdg_trace_apply(hdgdg_sim* sim, const double* x, double* y) {
    if (sim && explicit_scheme(&sim->cfg)) return fail(sim, HDGDG_EINVAL, "explicit scheme: no implicit stage");
    if (!sim || !x || !y) return fail(sim, HDGDG_EINVAL, "NULL argument to trace_apply");
    TRY(upload3(sim, sim->lam, x, sim->plan.nt));
    if (matrix_free(&sim->cfg)) {   // the handle's own operator: element by element, FP64-class
        CU(launch_mf_plain(sim->g, sim->mf, sim->lam, sim->gvec, beta_of(sim), sim->stream));
        return download(sim, y, sim->gvec, sim->plan.nt);
    }
    CU(launch_block_diag(sim->g, sim->Srr, sim->lam, sim->xt, sim->stream));          // u = S_rr x
    CU(launch_spmv_pre(sim->g, sim->Stil, sim->Scol, sim->xt, sim->gvec, sim->stream));  // y = S~ u
    return download(sim, y, sim->gvec, sim->plan.nt);
}

hdgdg_status hdgdg_set_trace_tile(hdgdg_sim* sim, int tile) {
    if (!sim) return fail(sim, HDGDG_EINVAL, "NULL handle");
    if (!matrix_free(&sim->cfg) || sim->ens)
        return fail(sim, HDGDG_EINVAL, "set_trace_tile: the handle has no matrix-free inner product");
    if (!mf_tile_ready(sim->g.P, tile))
        return fail(sim, HDGDG_EINVAL, "set_trace_tile: tile %d is not available at degree %d", tile, sim->g.P - 1);
    CU(cudaStreamSynchronize(sim->stream));
    for (auto& cg : sim->cycle_graph) drop_graph(sim, cg);   // the captured launches name the old tile
    drop_step_graphs(sim);
    sim->mf.tile = tile;
    if (tile == 0) sim->trace_tile = sim->trace_prefetch = 0;
    else mf_tile_info(sim->g.P, tile, &sim->trace_tile, &sim->trace_prefetch);
    return HDGDG_OK;
}

hdgdg_status hdgdg_set_local_tiles(hdgdg_sim* sim, int condense_tile, int recover_tile) {
    if (!sim) return fail(sim, HDGDG_EINVAL, "NULL handle");
    if (!sim->ops.schur || sim->ens)
        return fail(sim, HDGDG_EINVAL, "set_local_tiles: the handle's local solves are not the Schur kernels");
    for (int t : {condense_tile, recover_tile})
        if (!schur_tile_ready(sim->g.P, sim->ops.kind == 3, t))
            return fail(sim, HDGDG_EINVAL, "set_local_tiles: tile %d is not available at degree %d", t, sim->g.P - 1);
    CU(cudaStreamSynchronize(sim->stream));
    for (auto& cg : sim->cycle_graph) drop_graph(sim, cg);
    drop_step_graphs(sim);
    sim->ops.schur_tile_c = condense_tile;
    sim->ops.schur_tile_r = recover_tile;
    sim->ops.tile_condense = condense_tile == 0 ? 0 : schur_tile_epb(sim->g.P, condense_tile);
    sim->ops.tile_recover = recover_tile == 0 ? 0 : schur_tile_epb(sim->g.P, recover_tile);
    return HDGDG_OK;
}

hdgdg_status hdgdg_stage_solve(hdgdg_sim* sim, const double* R1, double* Q, double* qhat, int* iterations) {
    if (sim && explicit_scheme(&sim->cfg)) return fail(sim, HDGDG_EINVAL, "explicit scheme: no implicit stage");
    if (!sim || !R1 || !Q) return fail(sim, HDGDG_EINVAL, "NULL argument to stage_solve");
    const size_t n3 = 3 * sim->plan.n;
    TRY(upload3(sim, sim->R1, R1, n3));
    int its = 0;
    TRY(stage_solve_dev(sim, sim->R1, sim->Qs, sim->Ls[0], &its, sim->t));
    if (iterations) *iterations = its;
    TRY(download(sim, Q, sim->Qs, n3));
    if (qhat) TRY(download(sim, qhat, sim->lam, sim->plan.nt));
    return HDGDG_OK;
}

hdgdg_status hdgdg_set_kernel_timing(hdgdg_sim* sim, int on) {
    if (!sim) return HDGDG_EINVAL;
    TRY(sync(sim));
    sim->timing = on != 0;
    for (int c = 0; c < HDGDG_KT_COUNT; ++c) { sim->kt_ms[c] = 0.0; sim->kt_n[c] = 0; }
    return HDGDG_OK;
}

hdgdg_status hdgdg_kernel_time(hdgdg_sim* sim, int cls, double* total_ms, long long* launches) {
    if (!sim || cls < 0 || cls >= HDGDG_KT_COUNT || !total_ms || !launches)
        return fail(sim, HDGDG_EINVAL, "bad argument to kernel_time");
    TRY(sync(sim));
    *total_ms = sim->kt_ms[cls];
    *launches = sim->kt_n[cls];
    return HDGDG_OK;
}

hdgdg_status hdgdg_measure_fp64_tflops(double* tflops) {
    if (!tflops) return HDGDG_EINVAL;
    return measure_fp64_fma(tflops) == cudaSuccess ? HDGDG_OK : HDGDG_ECUDA;
}

hdgdg_status hdgdg_measure_conversion_rates(double* hardware_per_s, double* integer_per_s) {
    if (!hardware_per_s || !integer_per_s) return HDGDG_EINVAL;
    return measure_conversions(hardware_per_s, integer_per_s) == cudaSuccess ? HDGDG_OK : HDGDG_ECUDA;
}

}  // extern "C"

// ---- uneven ensembles ---------------------------------------------------------------------------
// Members of different mesh sizes and degrees advanced together: the members are grouped by
// (N, k) into batched handles, which hold each group's geometry and operators; a super-handle
// holds the ensemble's vectors (the groups one after another) and runs the time step of Algorithm
// 1 as one replayed graph whose geometry-dependent kernels each walk every group in one persistent
// launch (EnsTable), while the stage combinations and the Krylov vector work cover the whole
// ensemble as one vector.  The trace systems form one block-diagonal system solved by one GMRES,
// so a member's result agrees with its lone run to the solver tolerance.
struct hdgdg_ensemble {
    hdgdg_sim* sup = nullptr;
    std::vector<hdgdg_sim*> groups;
    std::vector<int> member_group, member_pos;   // member -> (group, instance within the group)
    std::vector<std::vector<double>> phiB;       // per member: phi_B at its nodes (host)
    EnsHost host;
    EnsGroup* d_grp = nullptr;
    std::string err;
};

namespace {

hdgdg_status ens_fail(hdgdg_ensemble* E, hdgdg_status st, const char* msg) {
    if (E) E->err = msg;
    return st;
}

// The super-handle: vectors for the whole ensemble, no operators of its own.
hdgdg_status ens_super(hdgdg_ensemble* E, const hdgdg_config* base, size_t n_total, size_t nt_total,
                       int edges_total, void* stream) {
    hdgdg_sim* sim = new (std::nothrow) hdgdg_sim();
    if (!sim) return HDGDG_ENOMEM;
    E->sup = sim;
    sim->cfg = *base;
    sim->cfg.batch = 1;
    sim->cfg.dt_per_instance = nullptr;
    scheme_tables(base->scheme, sim->A, sim->At, sim->b, sim->bt, &sim->s);
    sim->a_ii = sim->At[1][1];
    Plan& p = sim->plan;
    p.n = n_total;
    p.nt = nt_total;
    p.m = restart_of(base);
    p.s = sim->s;
    sim->g = host_geom(2, base->degree_k);   // not used by the ensemble's launches
    if (stream) {
        sim->stream = static_cast<cudaStream_t>(stream);
    } else {
        CU(cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking));
        sim->own_stream = true;
    }
    for (double** v : {&sim->q, &sim->q_new, &sim->R1, &sim->Z, &sim->Qs}) TRY(dalloc(sim, v, 3 * p.n));
    for (int i = 0; i < p.s; ++i) {
        TRY(dalloc(sim, &sim->NLs[i], 3 * p.n));
        TRY(dalloc(sim, &sim->Ls[i], 3 * p.n));
        CU(cudaMemsetAsync(sim->NLs[i], 0, 3 * p.n * sizeof(double), sim->stream));
        CU(cudaMemsetAsync(sim->Ls[i], 0, 3 * p.n * sizeof(double), sim->stream));
    }
    for (double** v : {&sim->gvec, &sim->xt, &sim->lam, &sim->w, &sim->fface}) TRY(dalloc(sim, v, p.nt));
    for (int i = 0; i < p.s; ++i)
        for (int h = 0; h < guess_order(base); ++h) {
            TRY(dalloc(sim, &sim->xhist[i][h], p.nt));
            TRY(dalloc(sim, &sim->yhist[i][h], p.nt));
        }
    TRY(dalloc(sim, &sim->V32, (size_t)(p.m + 1) * p.nt));
    TRY(dalloc(sim, &sim->w32, p.nt));
    TRY(dalloc(sim, &sim->red, reduction_scratch_doubles(p.m, edges_total, 3)));
    CU(cudaMemset(sim->red, 0, sizeof(double)));
    TRY(dalloc(sim, &sim->mred, mass_scratch_doubles()));
    TRY(dalloc(sim, &sim->dvals, 4 * (size_t)(p.m + 2) + 16));
    TRY(dalloc(sim, &sim->flags, 16));
    TRY(dalloc(sim, &sim->ctl, 1));
    TRY(dalloc(sim, &sim->sctl, 1));
    TRY(dalloc(sim, &sim->sstats, 1));
    TRY(dalloc(sim, &sim->dhist, kMaxStages));
    CU(cudaMallocHost(&sim->hhist, kMaxStages * sizeof(DevHist)));
    TRY(dalloc(sim, &sim->dls, kLsSlots));
    CU(cudaMallocHost(&sim->hbuf, (4 * (size_t)(p.m + 2) + 16) * sizeof(double)));
    CU(cudaStreamCreateWithFlags(&sim->body_stream, cudaStreamNonBlocking));
    double *ybuf = nullptr, *hm = nullptr, *hp = nullptr;
    TRY(dalloc(sim, &ybuf, p.nt));
    TRY(dalloc(sim, &hm, p.nt));
    TRY(dalloc(sim, &hp, p.nt));
    sim->mf.ybuf = ybuf;
    sim->mf.hm = hm;
    sim->mf.hp = hp;
    CU(cudaMemsetAsync(sim->flags, 0, 16, sim->stream));
    CU(cudaStreamSynchronize(sim->stream));
    return HDGDG_OK;
}

}  // namespace

extern "C" {

hdgdg_status hdgdg_ensemble_create(const hdgdg_config* base, int n_members, const int* n_side, const int* degree_k,
                                   const double* dt, const double* const* bottom_b, void* cuda_stream,
                                   hdgdg_ensemble** out) {
    if (!out) return HDGDG_EINVAL;
    *out = nullptr;
    if (!base || n_members < 1 || !n_side || !degree_k || !dt) return HDGDG_EINVAL;
    if (base->precision != HDGDG_MIXED || base->local_precision != HDGDG_LOCAL_F32X2 || base->trace_operator != 1 ||
        base->local_dense || (base->scheme != HDGDG_ARS2 && base->scheme != HDGDG_ARS3) ||
        base->boundary != HDGDG_PERIODIC || base->linear_only)
        return HDGDG_EINVAL;
    hdgdg_ensemble* E = new (std::nothrow) hdgdg_ensemble();
    if (!E) return HDGDG_ENOMEM;
    *out = E;
    // groups of equal (N, k), in order of first appearance
    std::vector<std::pair<int, int>> keys;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n_members; ++i) {
        if (n_side[i] < 2 || degree_k[i] < 2 || degree_k[i] > 4 || !(dt[i] > 0.0) || !std::isfinite(dt[i]))
            return ens_fail(E, HDGDG_EINVAL, "ensemble members need N >= 2, 2 <= k <= 4 and dt > 0");
        int gi = -1;
        for (size_t k = 0; k < keys.size(); ++k)
            if (keys[k].first == n_side[i] && keys[k].second == degree_k[i]) gi = (int)k;
        if (gi < 0) {
            if ((int)keys.size() == kEnsMaxGroups) return ens_fail(E, HDGDG_EINVAL, "more than 32 (N, k) groups");
            keys.push_back({n_side[i], degree_k[i]});
            members.emplace_back();
            gi = (int)keys.size() - 1;
        }
        E->member_group.push_back(gi);
        E->member_pos.push_back((int)members[gi].size());
        members[gi].push_back(i);
    }
    // one batched handle per group: geometry, bottoms, per-member time steps, operators
    size_t off3 = 0, offt = 0, n_total = 0, nt_total = 0;
    int edges_total = 0;
    E->phiB.resize(n_members);
    for (size_t gi = 0; gi < keys.size(); ++gi) {
        const int N = keys[gi].first, k = keys[gi].second, B = (int)members[gi].size();
        const size_t Np = (size_t)(k + 1) * (k + 1), nel = (size_t)N * N;
        std::vector<double> bot(B * nel * Np, 0.0), dts(B);
        double dtmax = 0.0;
        for (int j = 0; j < B; ++j) {
            const int m = members[gi][j];
            dts[j] = dt[m];
            dtmax = std::max(dtmax, dt[m]);
            if (bottom_b && bottom_b[m]) std::memcpy(&bot[j * nel * Np], bottom_b[m], nel * Np * sizeof(double));
            E->phiB[m].resize(nel * Np);
            for (size_t t = 0; t < nel * Np; ++t) E->phiB[m][t] = base->g * (base->H0 - bot[j * nel * Np + t]);
        }
        hdgdg_config c = *base;
        c.n_side = N;
        c.degree_k = k;
        c.batch = B;
        c.dt = dtmax;
        c.dt_per_instance = dts.data();
        c.host_steps = 1;
        hdgdg_sim* gs = nullptr;
        const hdgdg_status st = hdgdg_create(&c, bot.data(), cuda_stream, &gs);
        E->groups.push_back(gs);
        if (st != HDGDG_OK) return ens_fail(E, st, gs ? gs->err.c_str() : "group create failed");
        EnsGroup& G = E->host.h[gi];
        G.g = gs->g;
        G.off3 = off3;
        G.offt = offt;
        G.dt = gs->cfg.dt;
        G.beta = beta_of(gs);
        G.phiB = gs->phiB;
        G.tau = gs->tau;
        G.S2 = gs->ops.S;
        G.aux2 = gs->ops.aux;
        G.EG2 = gs->ops.EG;
        G.S32 = gs->mf.S32;
        G.aux32 = gs->mf.aux32;
        G.EG32 = gs->mf.EG32;
        G.Minv = gs->mf.Minv;
        off3 += 3 * gs->plan.n;
        offt += gs->plan.nt;
        n_total += gs->plan.n;
        nt_total += gs->plan.nt;
        edges_total += gs->g.n_edges;
    }
    E->host.ngroups = (int)keys.size();
    hdgdg_status st = ens_super(E, base, n_total, nt_total, edges_total, cuda_stream);
    if (st != HDGDG_OK) return ens_fail(E, st, E->sup ? E->sup->err.c_str() : "ensemble vectors");
    if (cudaMalloc(&E->d_grp, E->host.ngroups * sizeof(EnsGroup)) != cudaSuccess) {
        cudaGetLastError();
        return ens_fail(E, HDGDG_ENOMEM, "ensemble group table");
    }
    if (cudaMemcpy(E->d_grp, E->host.h, E->host.ngroups * sizeof(EnsGroup), cudaMemcpyHostToDevice) != cudaSuccess)
        return ens_fail(E, HDGDG_ECUDA, "ensemble group table copy");
    E->host.d_grp = E->d_grp;
    E->sup->ens = &E->host;
    return HDGDG_OK;
}

void hdgdg_ensemble_destroy(hdgdg_ensemble* E) {
    if (!E) return;
    if (E->sup) hdgdg_destroy(E->sup);
    for (hdgdg_sim* g : E->groups) hdgdg_destroy(g);
    if (E->d_grp) cudaFree(E->d_grp);
    delete E;
}

const char* hdgdg_ensemble_last_error(const hdgdg_ensemble* E) {
    if (!E) return "no ensemble";
    if (!E->err.empty()) return E->err.c_str();
    return E->sup ? E->sup->err.c_str() : "";
}

hdgdg_status hdgdg_ensemble_set_state(hdgdg_ensemble* E, int member, const double* h, const double* hu,
                                      const double* hv) {
    if (!E || !E->sup || member < 0 || member >= (int)E->member_group.size() || !h || !hu || !hv)
        return ens_fail(E, HDGDG_EINVAL, "bad argument to ensemble_set_state");
    const EnsGroup& G = E->host.h[E->member_group[member]];
    const size_t nm = (size_t)G.g.n_el_inst * G.g.Np, ng = (size_t)G.g.n_el * G.g.Np;
    const double gacc = E->sup->cfg.g;
    const std::vector<double>& pb = E->phiB[member];
    std::vector<double> q(3 * nm);
    for (size_t t = 0; t < nm; ++t) {
        const double phi = gacc * h[t];
        const double U = gacc * hu[t], V = gacc * hv[t];
        if (!std::isfinite(phi) || !std::isfinite(U) || !std::isfinite(V) || !(phi > 0.0))
            return ens_fail(E, HDGDG_ENONFINITE, "state has a non-finite value or non-positive depth");
        q[t] = phi - pb[t];
        q[nm + t] = U;
        q[2 * nm + t] = V;
    }
    hdgdg_sim* sim = E->sup;
    const size_t base = G.off3 + (size_t)E->member_pos[member] * nm;
    for (int c = 0; c < 3; ++c)
        CU(cudaMemcpyAsync(sim->q + base + c * ng, q.data() + c * nm, nm * sizeof(double), cudaMemcpyHostToDevice,
                           sim->stream));
    CU(cudaStreamSynchronize(sim->stream));
    sim->have_state = true;
    sim->stats = hdgdg_stats{};
    sim->t = 0.0;
    for (int i = 0; i < kMaxStages; ++i) sim->n_hist[i] = 0;   // the ensemble's solver history starts afresh
    return HDGDG_OK;
}

hdgdg_status hdgdg_ensemble_get_state(hdgdg_ensemble* E, int member, double* h, double* hu, double* hv) {
    if (!E || !E->sup || member < 0 || member >= (int)E->member_group.size() || !h || !hu || !hv)
        return ens_fail(E, HDGDG_EINVAL, "bad argument to ensemble_get_state");
    const EnsGroup& G = E->host.h[E->member_group[member]];
    const size_t nm = (size_t)G.g.n_el_inst * G.g.Np, ng = (size_t)G.g.n_el * G.g.Np;
    hdgdg_sim* sim = E->sup;
    std::vector<double> q(3 * nm);
    const size_t base = G.off3 + (size_t)E->member_pos[member] * nm;
    for (int c = 0; c < 3; ++c)
        CU(cudaMemcpyAsync(q.data() + c * nm, sim->q + base + c * ng, nm * sizeof(double), cudaMemcpyDeviceToHost,
                           sim->stream));
    CU(cudaStreamSynchronize(sim->stream));
    const double gacc = sim->cfg.g;
    const std::vector<double>& pb = E->phiB[member];
    for (size_t t = 0; t < nm; ++t) {
        h[t] = (q[t] + pb[t]) / gacc;
        hu[t] = q[nm + t] / gacc;
        hv[t] = q[2 * nm + t] / gacc;
    }
    return HDGDG_OK;
}

hdgdg_status hdgdg_ensemble_step(hdgdg_ensemble* E, int n_steps) {
    if (!E || !E->sup) return HDGDG_EINVAL;
    return hdgdg_step(E->sup, n_steps);
}

hdgdg_status hdgdg_ensemble_get_stats(hdgdg_ensemble* E, hdgdg_stats* out) {
    if (!E || !E->sup || !out) return ens_fail(E, HDGDG_EINVAL, "bad argument to ensemble_get_stats");
    *out = E->sup->stats;
    out->mass = 0.0;   // (per-member masses: hdgdg_ensemble_get_state; the ensemble reports none)
    return HDGDG_OK;
}

}  // extern "C"
