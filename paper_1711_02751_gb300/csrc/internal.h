// Internal declarations shared by the translation units of libhdgdg (not part of the ABI).
//
// Data layout in device memory (FP64):
//   state / stage vectors   [field c (phi_eta, U, V)][element e][node n = j*P + i]
//   trace vectors           [edge r][field c][node b]                (n_f = 3P per edge)
//   A^{-1} per element      [e][column s][row r], r, s = c*P*P + j*P + i  (column major)
//   preconditioned trace    [edge][slot 0..5][column jj][row ii]  of S~ = S M^{-1},
//     matrix (off-diagonal    slot order: the three other faces of the edge's minus
//     blocks only; the        element (ascending local face), then those of its plus
//     diagonal block is I)    element; column edge index in Scol[edge][slot]
//   block-Jacobi blocks     [edge][column jj][row ii] of M^{-1} = S_rr^{-1} and of S_rr
//
// Local faces of an element: 0 = x-minus (left), 1 = x-plus (right), 2 = y-minus, 3 = y-plus.
// Edge r < N^2 is face 1 of element r; edge N^2 + r is face 3 of element r.  The element on
// face 1/3 is the edge's "minus" side (normal +x / +y), the element on face 0/2 its "plus" side.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

namespace hdgdg {

constexpr int kMaxP = 9;   // degree k <= 8

// Division by a divisor fixed at create.  A general integer division compiles to conversions
// between integer and floating point, which GB300 executes at its FP64 rate; this is the
// round-up multiply of Granlund and Montgomery ("Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> 1)) >> (l - 1) for t = the high word of n m, exact for every 32-bit n.
struct FastDiv {
    unsigned d = 1, m = 0;
    int l = 0;
    __host__ void set(unsigned div) {
        d = div;
        m = 0;
        l = 0;
        if (div <= 1) return;
        while ((1ull << l) < div) ++l;
        m = (unsigned)((((1ull << 32) * ((1ull << l) - div)) / div) + 1);
    }
    __host__ __device__ __forceinline__ int div(int n) const {   // n >= 0
        if (d == 1) return n;
        const unsigned u = (unsigned)n;
#ifdef __CUDA_ARCH__
        const unsigned t = __umulhi(u, m);
#else
        const unsigned t = (unsigned)(((unsigned long long)u * m) >> 32);
#endif
        return (int)((t + ((u - t) >> 1)) >> (l - 1));
    }
};

// Mesh and GLL tables, passed by value to kernels.
struct Geom {
    int N, P, Np, n_el, n_edges;   // n_el, n_edges: totals over all instances of the batch
    int batch;                     // instances of the same N x N mesh advanced together
    int n_el_inst, n_edges_inst;   // per instance
    const double* dt_scale;        // device [batch]: instance time step / config time step, or NULL
    int walls;                  // 0: periodic unit square; 1: a bounded square (walls or Dirichlet)
    int dirichlet;              // 1: boundary faces take the moving-vortex exact solution (Sec. 7.1)
    double x0;                  // domain [x0, x0 + N h]^2
    double gacc, H0;            // gravity and reference depth (flat bottom for the vortex)
    double vortex[5];           // beta, u_inf, v_inf, x_c, y_c of eq. tc_vortex_ic
    double xi[kMaxP];           // GLL nodes
    double h;                   // element size (domain length / N)
    double two_over_h;          // d(xi)/dx
    double inv_w0;              // 1 / w_0 (= 1 / w_k): face lift of the collocated mass matrix
    double J;                   // area Jacobian (h/2)^2
    double w[kMaxP];            // GLL weights
    double D[kMaxP * kMaxP];    // D[r*P + c] = l_c'(xi_r)
    double Dhat[kMaxP * kMaxP]; // Dhat[i*P + a] = (w_a / w_i) D[a*P + i]: weak-form volume lift
    FastDiv byN, byN1, by_el, by_edges;   // / N, / (N + 1), / n_el_inst, / n_edges_inst
};

__host__ __device__ inline int face_node(int f, int b, int P) {
    return f == 0 ? b * P : f == 1 ? b * P + P - 1 : f == 2 ? b : (P - 1) * P + b;
}

// Connectivity of the N x N mesh.  Periodic: edge r < N^2 is face 1 of element r and edge
// N^2 + r face 3 of element r.  Walls: x-edges ey*(N+1) + ix (ix = 0..N), y-edges
// N(N+1) + iy*N + ex (iy = 0..N); a face on a wall has no neighbour (-1).
__host__ __device__ inline int local_edge_of_face(int e, int f, const Geom& g) {
    const int N = g.N, ey = g.byN.div(e), ex = e - ey * N;
    if (g.walls) {
        const int nx = N * (N + 1);
        switch (f) {
            case 0: return ey * (N + 1) + ex;
            case 1: return ey * (N + 1) + ex + 1;
            case 2: return nx + ey * N + ex;
            default: return nx + (ey + 1) * N + ex;
        }
    }
    switch (f) {
        case 0: return ey * N + (ex == 0 ? N - 1 : ex - 1);
        case 1: return e;
        case 2: return N * N + (ey == 0 ? N - 1 : ey - 1) * N + ex;
        default: return N * N + e;
    }
}

__host__ __device__ inline int local_neighbour(int e, int f, const Geom& g) {
    const int N = g.N, ey = g.byN.div(e), ex = e - ey * N;
    if (g.walls) {
        switch (f) {
            case 0: return ex > 0 ? e - 1 : -1;
            case 1: return ex < N - 1 ? e + 1 : -1;
            case 2: return ey > 0 ? e - N : -1;
            default: return ey < N - 1 ? e + N : -1;
        }
    }
    switch (f) {
        case 0: return ey * N + (ex == 0 ? N - 1 : ex - 1);
        case 1: return ey * N + (ex == N - 1 ? 0 : ex + 1);
        case 2: return (ey == 0 ? N - 1 : ey - 1) * N + ex;
        default: return (ey == N - 1 ? 0 : ey + 1) * N + ex;
    }
}

// Minus side (face 1 or 3: normal +x / +y) and plus side (face 0 or 2) of edge r; an absent
// side (wall) is -1 with the face it would have had.
__host__ __device__ inline void local_edge_sides(int r, const Geom& g, int* em, int* fm, int* ep, int* fp) {
    const int N = g.N;
    if (g.walls) {
        const int nx = N * (N + 1);
        if (r < nx) {
            const int ey = g.byN1.div(r), ix = r - ey * (N + 1);
            *em = ix >= 1 ? ey * N + ix - 1 : -1;
            *ep = ix < N ? ey * N + ix : -1;
            *fm = 1;
            *fp = 0;
        } else {
            const int rr = r - nx, iy = g.byN.div(rr), ex = rr - iy * N;
            *em = iy >= 1 ? (iy - 1) * N + ex : -1;
            *ep = iy < N ? iy * N + ex : -1;
            *fm = 3;
            *fp = 2;
        }
        return;
    }
    if (r < N * N) { *em = r; *fm = 1; *ep = local_neighbour(r, 1, g); *fp = 0; }
    else { const int e = r - N * N; *em = e; *fm = 3; *ep = local_neighbour(e, 3, g); *fp = 2; }
}

// Batched indices: instance i owns elements [i n_el_inst, (i+1) n_el_inst) and edges
// [i n_edges_inst, (i+1) n_edges_inst); connectivity never crosses instances.
__host__ __device__ inline int edge_of_face(int e, int f, const Geom& g) {
    const int inst = g.by_el.div(e);
    return inst * g.n_edges_inst + local_edge_of_face(e - inst * g.n_el_inst, f, g);
}

__host__ __device__ inline int neighbour(int e, int f, const Geom& g) {
    const int inst = g.by_el.div(e);
    const int nb = local_neighbour(e - inst * g.n_el_inst, f, g);
    return nb < 0 ? -1 : inst * g.n_el_inst + nb;
}

__host__ __device__ inline void edge_sides(int r, const Geom& g, int* em, int* fm, int* ep, int* fp) {
    const int inst = g.by_edges.div(r);
    local_edge_sides(r - inst * g.n_edges_inst, g, em, fm, ep, fp);
    if (*em >= 0) *em += inst * g.n_el_inst;
    if (*ep >= 0) *ep += inst * g.n_el_inst;
}

// Time-step factor of the instance that owns element e (1 without a batch table).
__host__ __device__ inline double dt_factor(const Geom& g, int e) {
    return g.dt_scale ? g.dt_scale[g.by_el.div(e)] : 1.0;
}

// The moving vortex of Sec. 7.1 (eq. tc_vortex_ic) at (x, y, t) as (phi_eta, U, V) over the
// flat bottom B = H0: H = H0 - beta^2/(16 pi^2 g) e^{-2(r^2-1)} (the printed beta^2/(32 pi^2) at
// g = 2), u = u_inf - beta/(2 pi) e^{-(r^2-1)} y_t, v = v_inf + beta/(2 pi) e^{-(r^2-1)} x_t.
__host__ __device__ inline void vortex_state(const Geom& g, double x, double y, double t, double* ph,
                                             double* U, double* V) {
    const double pi = 3.14159265358979323846;
    const double beta = g.vortex[0];
    const double xt = x - g.vortex[3] - g.vortex[1] * t;
    const double yt = y - g.vortex[4] - g.vortex[2] * t;
    const double e = exp(-(xt * xt + yt * yt - 1.0));
    const double H = g.H0 - beta * beta / (16.0 * pi * pi * g.gacc) * e * e;
    const double u = g.vortex[1] - beta / (2.0 * pi) * e * yt;
    const double v = g.vortex[2] + beta / (2.0 * pi) * e * xt;
    *ph = g.gacc * (H - g.H0);
    *U = g.gacc * H * u;
    *V = g.gacc * H * v;
}

// Physical coordinates of face node b of face f of element e.
__host__ __device__ inline void face_node_xy(const Geom& g, int e, int f, int b, double* x, double* y) {
    const int n = face_node(f, b, g.P), i = n % g.P, j = n / g.P;
    const int el = e - g.by_el.div(e) * g.n_el_inst, ey = g.byN.div(el);
    *x = g.x0 + (el - ey * g.N + 0.5 * (1.0 + g.xi[i])) * g.h;
    *y = g.x0 + (ey + 0.5 * (1.0 + g.xi[j])) * g.h;
}

// Host-built periodic unit-square mesh and GLL tables of an N x N, degree-k mesh (no GPU call).
Geom host_geom(int N, int k);

// Kernels launched by this library since load (every launcher adds its own launches).
long long launches_total();
void count_launches(int n);

// ---- kernel launchers (each returns the launch error) -------------------------------
// out = scale * M^{-1} NL(q); fface: scratch of n_edges * 3P doubles for the face fluxes
// t: time of the boundary data (Dirichlet boundaries only)
cudaError_t launch_dg_nl(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                         double scale, double* fface, double* out, cudaStream_t s, double t = 0.0);
// the same residual computed in FP32 arithmetic (FP64 storage): the mixed form's DG residual
// The mixed form's residual on FP32 copies (launch_dg_nl_f32 term for term): phi_B, tau and the
// face fluxes in FP32, the state in FP32 (q32, when given: the recovery's FP32 stage values) or
// FP64 (q64).
// fin (given, base set): the step's final update q_new = base + sum_k t.c[k] t.X[k] is formed by
// the element pass, term by term as launch_combine forms it, with this residual as term `slot`
// (t.X[slot] is not read); q_new goes to fin->qn, a non-finite entry sets *fin->nonfinite, and
// the residual itself is not written (out unused).  At most kFinalTerms terms.
constexpr int kFinalTerms = 4;
struct FinalSource;   // below, after CombineTerms
cudaError_t launch_dg_nl_f32io(const Geom& g, const double* q64, const float* q32, const float* phiB32,
                               const float* tau32, double scale, float* fface32, double* out, cudaStream_t s,
                               double t, const FinalSource* fin = nullptr);
cudaError_t launch_dg_nl_f32(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                             double scale, double* fface, double* out, cudaStream_t s, double t = 0.0);
// the same residual with its inputs (state, phi_B, tau) rounded to BF16 and FP32 arithmetic (k <= 4)
cudaError_t launch_dg_nl_bf16(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                              double scale, double* fface, double* out, cudaStream_t s, double t = 0.0);
// out = scale * M^{-1} (the explicit DG residual of the whole flux with the source term)
cudaError_t launch_dg_full(const Geom& g, const double* q, const double* phiB, double scale,
                           double* fface, double* out, cudaStream_t s, double t = 0.0);

struct CombineTerms {
    const double* X[10];
    double c[10];
    int n;
};
struct FinalSource {   // launch_dg_nl_f32io's final update
    const double* base = nullptr;
    CombineTerms t{};
    int slot = -1;
    double* qn = nullptr;
    unsigned* nonfinite = nullptr;
};
// out = base + sum_t c_t X_t over n doubles (out may alias base)
cudaError_t launch_combine(size_t n, const double* base, const CombineTerms& t, double* out,
                           unsigned* nonfinite_flag, cudaStream_t s);

// Setup: per element A^{-1} (column major) and the element Schur block S_e (pointwise rows).
cudaError_t launch_build_local(const Geom& g, const double* phiB, const double* tau_edge,
                               double dta, double* Ainv, double* Se, int* singular, cudaStream_t s);
// Setup: edge-block rows of S from S_e, S_rr^{-1}, S~ = S M^{-1} and the column indices.
cudaError_t launch_assemble_trace(const Geom& g, const double* Se, double* S7, double* Srr,
                                  double* Minv, double* Stil, int* Scol, int* singular,
                                  cudaStream_t s);

// The local operators as the condensation and recovery kernels apply them.
struct LocalOps {
    int kind = 0;                   // 0: per-element FP64; 1: per-element FP32; 2: shared, tensor cores;
                                    // 3: per-element FP32 pairs (FP64-class, compensated dot products);
                                    // 4: shared, tensor cores on BF16 slices (FP64-class)
    const double* Ainv = nullptr;   // kind 0: [n_el][col s][row r] = (A^{-1})_{rs}
    const float* Ainv32 = nullptr;  // kind 1: same layout in FP32
    const float* Ahi = nullptr;     // kind 3: A^{-1} = Ahi + Alo, same layout
    const float* Alo = nullptr;
    int tile_condense = 0, tile_recover = 0;              // kind 3: elements per block (0: default)
    int tile_condense_index = 0, tile_recover_index = 0;  // their index in the candidate list
    const void* image = nullptr;    // kind 2: the shared A^{-1} as a BF16 tensor-core operand tile
    int* error = nullptr;           // kinds 2, 4 and the staged Schur tile: set when a bounded wait ran out
    // Kinds 0 and 3 with schur set: A^{-1} applied through the Schur complement on phi.  Only the
    // (phi, phi) block of A^{-1} is kept, S [n_el][col m][row n], with aux [n_el][4][Np] =
    // (1/d, -cx, -cy, phi_B) per node and EG [batch][2][P][P] = (-E, -G) per instance; the values
    // are double (kind 0) or FP32 pairs float2 (hi, lo) (kind 3).
    bool schur = false;
    int schur_tile_c = 0, schur_tile_r = 0;   // tiles of the Schur kernels (launch_autotune_local)
    const void* S = nullptr;
    const void* aux = nullptr;
    const void* EG = nullptr;
};
// Whether tile t of the Schur kernels runs at degree P - 1 (pairs: FP32-pair operators), and its
// elements per block.
bool schur_tile_ready(int P, bool pairs, int t);
int schur_tile_epb(int P, int t);
// Setup of the Schur-complement local operators (LocalOps::S, aux, EG) from the FP64 A^{-1}, as
// double or, with f32x2, as FP32 pairs (float2).  dta = dt a_ii.
cudaError_t launch_schur_setup(const Geom& g, const double* Ainv, const double* phiB, const double* tau_edge,
                               double dta, bool f32x2, void* S, void* aux, void* EG, cudaStream_t s);
// Condensation: Z = A^{-1} R1 per element, then g = -C Z edge by edge (pointwise rows).
// t: time of the prescribed boundary traces (Dirichlet boundaries only)
// The stage's right-hand side formed inside the condensation (the Schur-complement kernels):
// R1 = base + sum_k t.c[k] t.X[k], term by term as launch_combine, written to R1 as it is read;
// at most kR1FusedTerms terms (an ARS2 stage has three).
constexpr int kR1FusedTerms = 4;
struct R1Source {
    const double* base = nullptr;   // nullptr: R1 is read as it stands
    CombineTerms t{};
};
cudaError_t launch_condense(const Geom& g, const LocalOps& ops, const double* R1, const double* phiB,
                            const double* tau_edge, double* Z, double* gvec, cudaStream_t s, double t = 0.0,
                            const R1Source* src = nullptr);
// Recovery: Q = Z + beta A^{-1} (tau qhat) on boundary nodes; Lst = (Q - R1) / a_ii.
// Lst = (Q - R1) inv_aii; the Schur-complement kinds take inv_aii = 1 only (cudaErrorInvalidValue
// otherwise): the time step keeps Q - R1 and folds 1/a_ii into its combinations.
cudaError_t launch_recover(const Geom& g, const LocalOps& ops, const double* Z, const double* R1,
                           const double* tau_edge, const double* qhat, double beta, double inv_aii,
                           double* Q, double* Lst, cudaStream_t s, float* Q32 = nullptr);
// Autotuner of the local kernels' tile (elements per block): times each candidate on the handle's
// operators, using R1, Z, Q, Lst as scratch (their contents are overwritten), and records the
// fastest in ops: the Schur-complement kernels (FP64 or FP32 pairs, degrees 2..4) and the dense
// FP32-pair kernels.  No-op for other local arithmetic.
cudaError_t launch_autotune_local(const Geom& g, LocalOps& ops, double* R1, double* Z, const double* tau_edge,
                                  const double* qhat, double* Q, double* Lst, cudaStream_t s);
// The block-Jacobi inverse of the matrix-free operator: per edge its NF x NF block (column major) as
// FP16 values of the block divided by a power of two, and that power of two (the block's scale).
// The values are the preconditioner -- every use (inner cycles, refinement residual,
// back-transformation) reads these same numbers.
struct PrecondBlocks {
    const __half* h = nullptr;
    const float* scale = nullptr;
};
// Matrix-free trace operator (kernels_mf.cu): S x = D x - C A^{-1} B x element by element through
// the Schur-complement local solve, with the block-Jacobi preconditioner M^{-1} applied first.
struct MfOps {
    const float *S32 = nullptr, *aux32 = nullptr, *EG32 = nullptr;   // Schur operators, FP32 (inner cycles)
    const void *S2 = nullptr, *aux2 = nullptr, *EG2 = nullptr;       // the same as FP32 pairs (float2)
    PrecondBlocks Minv;              // block-Jacobi inverse [edge][col][row], FP16 with a scale per edge
    const double* tau = nullptr;     // tau_hat [edge][P]
    const float* tau32 = nullptr;    // the same rounded to FP32 (the inner cycles' fused pass)
    const void* tau2 = nullptr;      // and as FP32 pairs (float2; the refinement residual)
    void* ybuf = nullptr;            // scratch: M^{-1} x (n_edges * 3P values of 8 bytes)
    void* hm = nullptr;              // scratch: the edges' minus-side halves of S y (8 bytes per value)
    void* hp = nullptr;              // scratch: their plus-side halves
    int tile = 0;                    // tile of the inner cycles' element pass (launch_mf_autotune)
    int tile_res = 0;                // tile of the refinement residual's element pass
};
// y = S M^{-1} x in FP32 (inner Krylov cycles), one fused launch that adds into y; done as for
// launch_spmv_pre.  y_zeroed: the caller guarantees y = 0 (else a zeroing launch comes first).
// With 3(k + 1) a multiple of 4, x must start on 16 bytes (cudaErrorMisalignedAddress otherwise).
cudaError_t launch_mf_inner(const Geom& g, const MfOps& op, const float* x, float* y, double beta, cudaStream_t s,
                            const int* done = nullptr, bool y_zeroed = false);
// w = rhs - S M^{-1} x in FP64-class FP32-pair arithmetic (the refinement's true residual); with
// nrm_scratch (a reduction scratch, as launch_multidot's) also ||w||^2 into *nrm_out, in the last pass
cudaError_t launch_mf_residual(const Geom& g, const MfOps& op, const double* x, const double* rhs, double* w,
                               double beta, cudaStream_t s, double* nrm_scratch = nullptr, double* nrm_out = nullptr);
// w = rhs - (hm + hp) and ||w||^2 (16-byte aligned vectors; cudaErrorMisalignedAddress otherwise)
cudaError_t launch_sum_residual_norm(size_t n, const double* hm, const double* hp, const double* rhs, double* w,
                                     double* scratch, double* out, cudaStream_t s);
// y = S x (no preconditioner), FP64-class
cudaError_t launch_mf_plain(const Geom& g, const MfOps& op, const double* x, double* y, double beta, cudaStream_t s);
// Whether tile t of the inner element pass can run at degree P - 1, and its elements per block and
// whether it loads the S^{-1} row into registers ahead of the traces.
bool mf_tile_ready(int P, int t);
void mf_tile_info(int P, int t, int* epb, int* prefetch);
// Pick the inner element pass's tile by timing each candidate (degrees 2..4); *epb and *prefetch
// report the choice (elements per block, S^{-1} row in registers).
cudaError_t launch_mf_autotune(const Geom& g, MfOps& op, const float* x, float* y, const double* xd,
                               const double* rhs, double* w, double beta, cudaStream_t s, int* epb, int* prefetch);
// qhat = M^{-1} x~ with the FP32 blocks, FP64-class sums
cudaError_t launch_mf_back(const Geom& g, const PrecondBlocks& M, const double* x, double* y, cudaStream_t s);
// The FP16 blocks and scales from the FP64 block-Jacobi inverse (setup).
cudaError_t launch_precond_f16(const double* Minv, int n_edges, int NF, __half* h, float* scale, cudaStream_t s);
// hi[t] = pairs[t].x for n FP32 pairs (float2)
cudaError_t launch_pair_hi(const void* pairs, float* hi, size_t n, cudaStream_t s);
// hi = (float)a, lo = (float)(a - hi): the FP32-pair copy of an FP64 array.
cudaError_t launch_split_f32x2(const double* a, float* hi, float* lo, size_t n, cudaStream_t s);
// Tensor-core tile of one shared operator: bytes of the BF16 image, and its build from the
// FP64 A^{-1} of element 0 (setup).
size_t tc_image_bytes(int P);
cudaError_t launch_tc_image(const Geom& g, const double* Ainv, void* image, cudaStream_t s);
// The FP64-class variant: the operator as five seven-bit BF16 slices with column exponents (the
// Ozaki splitting), its image bytes and build; the products of the slices on the tensor cores.
size_t tc_split_image_bytes(int P);
cudaError_t launch_tc_split_image(const Geom& g, const double* Ainv, void* image, cudaStream_t s);
cudaError_t launch_local_tc_split(const Geom& g, int mode, const void* image, const double* R1, const double* Z,
                                  const double* tau_edge, const double* qhat, double beta, double inv_aii,
                                  double* out0, double* out1, int* error, cudaStream_t s);
// Z = A^{-1} R1 (mode 0) or Q = Z + beta A^{-1}(tau qhat), Lst = (Q - R1)/a_ii (mode 1) on the
// tensor cores with the shared operator image.
cudaError_t launch_local_tc(const Geom& g, int mode, const void* image, const double* R1,
                            const double* Z, const double* tau_edge, const double* qhat, double beta,
                            double inv_aii, double* out0, double* out1, int* error, cudaStream_t s);

// Krylov set on trace vectors of n = n_edges * nf values.  Overloads on the storage type:
// double for the FP64 path, float for the inner solves of the mixed-precision path.
// y = x + sum_slots S~ x[col]   (S~ with identity diagonal blocks)
// done (may be NULL): device flag; the Krylov-loop kernels return at once when it is set.
cudaError_t launch_spmv_pre(const Geom& g, const double* Stil, const int* Scol, const double* x,
                            double* y, cudaStream_t s, const int* done = nullptr);
// FP32: given stream_error (a device int set when a bounded wait runs out), the matrix is
// streamed through shared memory by bulk copies in a persistent pipelined kernel instead.
cudaError_t launch_spmv_pre(const Geom& g, const float* Stil, const int* Scol, const float* x,
                            float* y, cudaStream_t s, const int* done = nullptr, int* stream_error = nullptr);
// w = rhs - (x + S~ x) with S~ = Shi + Slo (FP32 pair, compensated sums) and ||w||^2 -> *nrm2 in
// one pass; scratch as for launch_multidot (a ticket counter and at least 2432 partial sums).
cudaError_t launch_residual_norm_x2(const Geom& g, const float* Shi, const float* Slo, const int* Scol,
                                    const double* x, const double* rhs, double* w, double* scratch, double* nrm2,
                                    cudaStream_t s);
// y = B x for a block-diagonal matrix B given as [edge][col][row] blocks: FP64, or (pairs) FP32
// pairs stored in the same eight bytes per entry (launch_split_pairs_inplace), compensated sums.
cudaError_t launch_block_diag(const Geom& g, const double* Bd, const double* x, double* y,
                              cudaStream_t s, bool pairs = false);
// a[i] -> (float hi, float lo) in place, as float2 (split of compensated.h)
cudaError_t launch_split_pairs_inplace(double* a, size_t n, cudaStream_t s);
// Device-resident control block of one GMRES(m) solve (m <= kM): Hessenberg matrix, Givens
// rotations, residual estimates and the stop flags the loop kernels test.
struct GmresCtl {
    static constexpr int kM = 32;
    double H[kM + 1][kM];
    double Hr[kM + 1][kM];   // the Hessenberg columns before the Givens rotations
    double cdl[kM + 1];      // H h2 of the last column (launch_dcgs_fused)
    double cs[kM], sn[kM], s[kM + 1], y[kM];
    double tol_abs;     // the solve stops when the residual estimate is <= tol_abs
    double inner_rel;   // a cycle also stops at inner_rel * (its starting residual); 0 = off
    double tol_cycle;
    double rnorm;       // residual norm at the start of the current cycle
    int done, jend, total, maxit, status;
};

// out[j] = <V_j, w>, j < nv, V_j = V + j * ldv; uses a scratch of dot_scratch_doubles(nv)
// doubles (a ticket counter, zero between calls, then the block partial sums) that every call
// on one stream may share.  Deterministic (fixed grid, fixed order).
size_t dot_scratch_doubles(int nv);
// The handle's reduction scratch: the Gram-Schmidt dots of a GMRES(m) cycle, the fused
// residual pass (launch_residual_norm_x2) and the guess norms (launch_guess_norms) share it.
size_t reduction_scratch_doubles(int m, int n_edges, int P);
// Candidate initial guesses of a trace solve: y[j] = S~ x~_{n-1-j} (j < nq) and the extrapolation
// coefficients of each order q = 1..nq.  out[0] = ||g||^2, out[q] = ||g - sum_j c[q][j] y[j]||^2.
struct GuessTerms {
    const double* y[6];
    double c[7][6];
    int nq;
};
size_t guess_scratch_doubles();
// f32x2 (the mixed form, whose tolerance is 1e-9 ||g||): the candidates formed in FP32 from the
// differences g - y_0 and y_0 - y_j taken from FP32 pairs -- each candidate norm to FP32 relative
// accuracy, enough to choose the start, whose norm the solve then takes exactly.
cudaError_t launch_guess_norms(size_t n, const double* g, const GuessTerms& t, double* scratch, double* out,
                               cudaStream_t s, bool f32x2 = false);
cudaError_t launch_multidot(const double* V, size_t ldv, int nv, const double* w, size_t n,
                            double* scratch, double* out, cudaStream_t s, const int* done = nullptr);
cudaError_t launch_multidot(const float* V, size_t ldv, int nv, const float* w, size_t n,
                            double* scratch, double* out, cudaStream_t s, const int* done = nullptr);
// Fused tail of classical Gram-Schmidt applied twice, given h1 = V^T w on the device:
// w1 = w - V h1 (in place), h2 = V^T w1, ||w1||^2 -> *nw1, hn = sqrt(||w1||^2 - ||h2||^2),
// vout = (w1 - V h2) / hn.  nv <= 32; scratch of dot_scratch_doubles(nv + 1).
// With a GMRES control block, column j of the Hessenberg matrix, its Givens rotation and the
// cycle's stop test are done in the same launch (restart length m).  twice = false: classical
// Gram-Schmidt once (h2 = 0, hn = ||w1||, vout = w1 / hn).
cudaError_t launch_cgs2_tail(const double* V, size_t ldv, int nv, const double* h1, double* w, size_t n,
                             double* scratch, double* h2, double* nw1, double* hn, double* vout,
                             GmresCtl* ctl, int j, int m, bool twice, cudaStream_t s, const int* done = nullptr);
// zero: a vector other than w set to 0 in the same pass (the next fused matrix-free product adds into it)
cudaError_t launch_cgs2_tail(const float* V, size_t ldv, int nv, const double* h1, float* w, size_t n,
                             double* scratch, double* h2, double* nw1, double* hn, float* vout,
                             GmresCtl* ctl, int j, int m, bool twice, cudaStream_t s, const int* done = nullptr,
                             float* zero = nullptr);
// Classical Gram-Schmidt twice with the second pass delayed (the FP32 inner cycles of the
// matrix-free form).  launch_cgs2_update: w1 = w - V h1 in place, h2 = V^T w1, hn = ||w1 - V h2||
// (for an orthonormal V), the Hessenberg column j with its rotation and stop test, and
// ctl->cdl = H h2 -- the second pass itself is left to launch_dcgs_fused, which, given the
// product z of w1, forms v = (w1 - V h2) / hn into vout, the product of v in place of w1, and
// V_k . (A v) for k <= nj into h1n (the next step's first pass); zero = 0 when given.  nj <= 31.
cudaError_t launch_cgs2_update(const float* V, size_t ldv, int nv, const double* h1, float* w, size_t n,
                               double* scratch, double* h2, double* nw1, double* hn, GmresCtl* ctl, int j, int m,
                               cudaStream_t s, const int* done);
cudaError_t launch_dcgs_fused(const float* V, size_t ldv, int nj, const double* h2, const double* hn,
                              const GmresCtl* ctl, float* w, const float* z, float* vout, float* zero, size_t n,
                              double* scratch, double* h1n, cudaStream_t s, const int* done);


// ---- uneven ensembles: one persistent launch per kernel class over many mesh groups ----------
// A group is a batch of instances of one mesh size and degree (its own geometry, operators and
// time step); the ensemble's vectors hold the groups one after another (group-major), each
// group's slice laid out as a lone handle's.  A launch covers every group: its work list is the
// concatenation of the groups' blocks, and a persistent grid walks it, each block taking items
// (group, block of that group) until the list is done.
constexpr int kEnsMaxGroups = 32;
struct EnsGroup {
    Geom g;                     // the group's mesh (a batch of same-size instances)
    size_t off3, offt;          // its slice: state vectors (3 fields), trace vectors
    double dt, beta;            // its time step and lift factor dt a_ii (2/h) / w_0
    const double* phiB;
    const double* tau;
    const void *S2, *aux2, *EG2;          // Schur-complement operators as FP32 pairs
    const float *S32, *aux32, *EG32;      // and as FP32 (the inner cycles)
    PrecondBlocks Minv;                   // block-Jacobi inverse, FP16 blocks and scales
};
struct EnsTable {               // one launch: the groups and the first work item of each
    const EnsGroup* grp;        // device array [ngroups]
    int ngroups;
    int start[kEnsMaxGroups + 1];
};
struct EnsHost {                // host copy of the group list, for building launch tables
    const EnsGroup* d_grp = nullptr;
    int ngroups = 0;
    EnsGroup h[kEnsMaxGroups];
};
// DG residual of the nonlinear part in FP32 arithmetic over every group (face pass, element pass)
cudaError_t launch_ens_dg_nl_f32(const EnsHost& E, const double* q, double* fface, double* out, cudaStream_t s);
// condensation: Z = A^{-1} R1 (FP32-pair Schur route), g = -C Z
cudaError_t launch_ens_condense(const EnsHost& E, const double* R1, double* Z, double* gvec, cudaStream_t s);
// recovery: Q = Z + beta A^{-1}(tau qhat), Lst = (Q - R1)/a_ii
cudaError_t launch_ens_recover(const EnsHost& E, const double* Z, const double* R1, const double* qhat,
                               double inv_aii, double* Q, double* Lst, cudaStream_t s);
// matrix-free trace operator over every group: inner (FP32), residual (FP32 pairs), back-transformation
cudaError_t launch_ens_mf_inner(const EnsHost& E, const MfOps& scratch, size_t nt, const float* x, float* y,
                                cudaStream_t s, const int* done);
cudaError_t launch_ens_mf_residual(const EnsHost& E, const MfOps& scratch, size_t nt, const double* x,
                                   const double* rhs, double* w, cudaStream_t s);
cudaError_t launch_ens_mf_back(const EnsHost& E, const double* x, double* y, cudaStream_t s);

// Whole-step graphs (kernels_ctl.cu): the trace solve's decisions taken on the device.
struct SolveCtl {
    double bnorm, tol, rnorm;
    int guess;    // extrapolation order the solve started from (0: zero)
    int active;   // 0 when g = 0 or not finite (nothing to solve)
};
struct StepStats {            // counters of one replayed step, read by the host after it
    long long its;            // GMRES iterations over the step's solves
    int last_its, last_guess, cycles;
    double last_rel;
    unsigned nonfinite, notconv;
    int notconv_its;
    double notconv_rel;
};
struct GuessHistory {         // the stage's stored solutions x~ and products S~x~, newest first
    const double* x[6];
    const double* y[6];
    double c[7][6];           // extrapolation coefficients of each order
};
// A stage's guess history as the replayed step graph reads it, from device memory: the host
// rotates its pointers after every step and copies this table before the replay, so one captured
// graph serves every rotation and history length.
struct DevHist {
    const double* x[6];   // stored solutions x~, newest first (the first `avail` are valid)
    const double* y[6];   // their products S~ x~
    double* xw;           // the slot this step's solution goes to (it becomes the newest)
    double* yw;
    int avail;            // candidates of the start (<= the extrapolation order)
    int has_history;      // avail > 0 (gates the plain norm of g, read as a `done` flag)
};
cudaError_t launch_solve_begin(const double* cand, int avail, double rtol, double inner_rel, int maxit, GmresCtl* ctl,
                               SolveCtl* sc, StepStats* ss, double* nrm2, cudaStream_t s);
cudaError_t launch_guess_apply(size_t n, const double* g, const GuessHistory& h, const SolveCtl* sc, double* xt,
                               double* w, cudaStream_t s);
// The same two steps with the history's length and pointers read from dh (the step graph's form).
cudaError_t launch_solve_begin_dev(const double* cand, const DevHist* dh, double rtol, double inner_rel, int maxit,
                                   GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double* nrm2, cudaStream_t s);
cudaError_t launch_guess_apply_dev(size_t n, const double* g, const DevHist* dh, const double (*coef)[6],
                                   const SolveCtl* sc, double* xt, double* w, cudaStream_t s);
// out[0..avail] = ||g||^2 and the candidates' squared residual norms (launch_guess_norms), for
// avail = dh->avail > 0; returns at once when there is no history.
cudaError_t launch_guess_norms_dev(size_t n, const double* g, const DevHist* dh, const double (*coef)[6],
                                   double* scratch, double* out, cudaStream_t s, bool f32x2);
// The least-squares start (krylov_guess_ls, mixed form): the Gram sums of the stored products'
// differences into ls[0..31] (launch_guess_gram: t.nq stored products; _dev: from dh), the
// small solve into ls[32..39] (zero start's and the projection's squared residuals, the affine
// coefficients alpha), and for the step graph the choice and its application.
cudaError_t launch_guess_gram(size_t n, const double* g, const GuessTerms& t, double* scratch, double* out,
                              cudaStream_t s);
cudaError_t launch_guess_gram_dev(size_t n, const double* g, const DevHist* dh, double* scratch, double* out,
                                  cudaStream_t s);
cudaError_t launch_ls_solve(double* ls, int avail, cudaStream_t s);
cudaError_t launch_ls_start_dev(size_t n, const double* g, const DevHist* dh, double* ls, double rtol,
                                double inner_rel, int maxit, GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double* nrm2,
                                double* xt, double* w, cudaStream_t s);
constexpr int kLsSlots = 40;
// dh->xw = xt, dh->yw = g - w (the solve's S~ x~ from its final true residual w)
cudaError_t launch_hist_store_dev(size_t n, const double* xt, const double* g, const double* w, const DevHist* dh,
                                  cudaStream_t s);
cudaError_t launch_loop_begin(double* nrm2, const double* nrm_exact, int use_exact, SolveCtl* sc, StepStats* ss,
                              cudaGraphConditionalHandle loop, cudaStream_t s);
cudaError_t launch_cycle_end(const double* nrm2, const GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double stagnation,
                             cudaGraphConditionalHandle loop, cudaStream_t s);
cudaError_t launch_solve_end(const GmresCtl* ctl, const SolveCtl* sc, StepStats* ss, cudaStream_t s);

cudaError_t launch_gmres_solve_init(GmresCtl* c, double tol_abs, double inner_rel, int maxit, cudaStream_t s);
cudaError_t launch_gmres_cycle_init(GmresCtl* c, const double* nrm2, cudaStream_t s);

// y = H^{-1} s, then x += V y (FP64 x; V of either type)
cudaError_t launch_gmres_update(const double* V, size_t ldv, GmresCtl* c, double* x, size_t n, cudaStream_t s);
cudaError_t launch_gmres_update(const float* V, size_t ldv, GmresCtl* c, double* x, size_t n, cudaStream_t s);
// v = w / sqrt(*nrm2), w in FP64
cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, double* v, size_t n,
                                  cudaStream_t s);
// (and zero = 0 when given: the output of the cycle's first fused matrix-free product)
cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, float* v, size_t n,
                                  cudaStream_t s, float* zero = nullptr);
cudaError_t launch_to_f32(const double* a, float* b, size_t n, cudaStream_t s);

// User-state conversion and diagnostics.
cudaError_t launch_user_to_state(const Geom& g, const double* h, const double* hu, const double* hv,
                                 const double* phiB, double gacc, double* q, unsigned* bad,
                                 cudaStream_t s);
cudaError_t launch_state_to_user(const Geom& g, const double* q, const double* phiB, double gacc,
                                 double* h, double* hu, double* hv, cudaStream_t s);
size_t mass_scratch_doubles();
cudaError_t launch_mass(const Geom& g, const double* q, double* scratch, double* out, cudaStream_t s);

cudaError_t measure_fp64_fma(double* tflops);
cudaError_t measure_conversions(double* hw_per_s, double* int_per_s);

}  // namespace hdgdg
