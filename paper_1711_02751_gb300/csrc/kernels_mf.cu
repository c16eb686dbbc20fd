// Matrix-free application of the condensed trace operator (eq. linearizedHDGsystem_schur):
//   S x = D x - C A^{-1} B x,
// computed element by element instead of through the assembled edge-block matrix.  With the
// pointwise rows of the conservation condition (eq. HDGcont divided by its face weight) the
// pieces are node-local:
//   -B x   lifts tau x onto the element's boundary nodes (corners take both faces) with the
//          factor beta = dt a_ii (2/h) / w_0 -- the same lift as the local recovery;
//   A^{-1} is the Schur-complement-on-phi solve of schur.h;
//   C W    at an edge node takes, from each side with outward normal n and W = (phi, U):
//          phi_hat row  U.n + tau phi,   momentum rows  phi_B phi n + tau U;
//   D      is -2 tau on every row (the two sides' -tau).
// A reflecting wall's absent side is the mirror of the present one (its C rows double the
// phi_hat and tangential terms and cancel the normal one), and a prescribed (Dirichlet) trace
// row is the identity -- the rows the assembled matrix holds.
//
// One thread per (element, node), EPB elements per block, as the local solves.  An edge's row
// needs both of its elements: each element leaves its half of the row in memory (the minus side
// in the output vector, the plus side in a scratch vector) and takes a ticket (one int per edge);
// the element that arrives second reads the other half and writes minus half + plus half, always
// in that order, so the result does not depend on which element came first.  Nothing waits: the
// first element's block simply moves on.
//
// Modes (the Krylov solve applies the block-Jacobi-preconditioned operator S~ = S M^{-1}):
//   kMfInner     y = S M^{-1} x        FP32 arithmetic and vectors (the mixed form's inner cycles)
//   kMfResidual  w = g - S M^{-1} x    FP64-class FP32-pair arithmetic, FP64 vectors (refinement)
//   kMfPlain     y = S x               FP64-class, FP64 vectors (the row-level entry point)
// M^{-1} is the block-Jacobi inverse held in FP32 [edge][col][row]; the residual and the final
// back-transformation qhat = M^{-1} x~ use exactly these FP32 values, so the preconditioner is
// the same matrix on every path.
#include <type_traits>

#include "compensated.h"
#include "internal.h"
#include "schur.h"

namespace hdgdg {
namespace {

enum MfMode { kMfInner = 0, kMfResidual = 1, kMfPlain = 2 };

// elements per block: 256 threads, at most 32 elements (the block's shared arrays stay under 48 KB)
template <int P>
constexpr int mf_epb() {
    return 256 / (P * P) > 32 ? 32 : (256 / (P * P) > 0 ? 256 / (P * P) : 1);
}

template <class A>
__device__ __forceinline__ typename A::T arith_of_f32(float v) {
    if constexpr (sizeof(typename A::T) == sizeof(float)) return v;
    else if constexpr (sizeof(typename A::T) == sizeof(float2)) return float2{v, 0.f};
    else return (double)v;
}

template <class A, typename TX>
__device__ __forceinline__ typename A::T arith_load(const TX* p) {
    if constexpr (sizeof(TX) == sizeof(float)) return arith_of_f32<A>(*p);
    else return A::from(*p);
}

template <int P, int EPB, class A>
struct MfSmem {
    using T = typename A::T;
    static constexpr int NF = 3 * P;
    SchurSmem<P, EPB, A> sc;
    T x[EPB][4][NF];     // the element's four face traces
    T y[EPB][4][NF];     // M^{-1} x of each face (x itself in plain mode)
    T h[EPB][4][NF];     // the element's half of each face's row of S y
    int ed[EPB][4];      // edge of each face
    int nb[EPB][4];      // neighbour across each face (-1: boundary)
    int second[EPB][4];  // 1 when this element completes the face's row
};

template <int P, int EPB, class A, int MODE>
__global__ void __launch_bounds__(EPB * P * P)
    mf_trace_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                    const typename A::T* __restrict__ EG, const float* __restrict__ Minv,
                    const double* __restrict__ tau_edge,
                    const std::conditional_t<MODE == kMfInner, float, double>* __restrict__ x,
                    const double* __restrict__ rhs,
                    std::conditional_t<MODE == kMfInner, float, double>* __restrict__ out,
                    std::conditional_t<MODE == kMfInner, float, double>* __restrict__ half,
                    int* __restrict__ ticket, double beta, const int* __restrict__ done) {
    using T = typename A::T;
    using TO = std::conditional_t<MODE == kMfInner, float, double>;
    constexpr int Np = P * P, NF = 3 * P, NFACE = 4 * NF;
    if (done && *done) return;
    __shared__ MfSmem<P, EPB, A> sm;
    const int le = threadIdx.x / Np, n = threadIdx.x % Np, i = n % P, j = n / P;
    const int e = blockIdx.x * EPB + le;
    const bool live = e < g.n_el;
    if (live && n < 4) {
        sm.ed[le][n] = edge_of_face(e, n, g);
        sm.nb[le][n] = neighbour(e, n, g);
    }
    __syncthreads();
    if (live) {
        for (int t = n; t < NFACE; t += Np) {
            const int f = t / NF, k = t % NF;
            sm.x[le][f][k] = arith_load<A>(x + (size_t)sm.ed[le][f] * NF + k);
        }
    }
    __syncthreads();
    if (live) {   // y = M^{-1} x, face by face
        for (int t = n; t < NFACE; t += Np) {
            const int f = t / NF, row = t % NF;
            if constexpr (MODE == kMfPlain) {
                sm.y[le][f][row] = sm.x[le][f][row];
            } else {
                const float* M = Minv + (size_t)sm.ed[le][f] * NF * NF + row;
                typename A::Acc acc;
#pragma unroll
                for (int col = 0; col < NF; ++col) acc.add(arith_of_f32<A>(__ldg(M + col * NF)), sm.x[le][f][col]);
                sm.y[le][f][row] = acc.get();
            }
        }
    }
    __syncthreads();
    // lift: u = sum over the faces through node n of tau y (the recovery's -B y / beta)
    T u[3];
    {
        typename A::Acc a0, a1, a2;
        if (live) {
            for (int f = 0; f < 4; ++f) {
                const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                                (f == 3 && j == P - 1);
                if (!on) continue;
                const int b = (f < 2) ? j : i;
                const T tau = A::from(tau_edge[(size_t)sm.ed[le][f] * P + b]);
                a0.add(tau, sm.y[le][f][b]);
                a1.add(tau, sm.y[le][f][P + b]);
                a2.add(tau, sm.y[le][f][2 * P + b]);
            }
        }
        u[0] = a0.get();
        u[1] = a1.get();
        u[2] = a2.get();
    }
    T W[3];
    schur_solve<P, EPB, A>(sm.sc, g, e, le, n, live, S, aux, EG, u[0], u[1], u[2], W[0], W[1], W[2]);
    if (live) {
        const T bt = A::from(beta * dt_factor(g, e));
        W[0] = A::mul(bt, W[0]);
        W[1] = A::mul(bt, W[1]);
        W[2] = A::mul(bt, W[2]);
        const T pb = aux[(size_t)e * 4 * Np + 3 * Np + n];
        const T one = A::from(1.0), mone = A::from(-1.0);
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const bool xedge = f < 2, minus = (f == 1 || f == 3);   // minus side: outward normal +axis
            const int cn = xedge ? 1 : 2, ct = xedge ? 2 : 1;
            const double tau_d = tau_edge[(size_t)sm.ed[le][f] * P + b];
            const T tau = A::from(tau_d), m2tau = A::from(-2.0 * tau_d);
            const T Wn = W[cn], Wt = W[ct];
            const T sg = minus ? one : mone;
            const bool boundary = sm.nb[le][f] < 0;
            if (boundary && g.dirichlet) {   // prescribed trace: the identity row
                sm.h[le][f][b] = sm.y[le][f][b];
                sm.h[le][f][P + b] = sm.y[le][f][P + b];
                sm.h[le][f][2 * P + b] = sm.y[le][f][2 * P + b];
                continue;
            }
            typename A::Acc r0, rn, rt;
            r0.add(sg, Wn);                       // U.n
            r0.add(tau, W[0]);                    // + tau phi
            rn.add(A::mul(sg, pb), W[0]);         // phi_B phi n
            rn.add(tau, Wn);                      // + tau U_n
            rt.add(tau, Wt);                      // tau U_t
            if (boundary) {                       // wall: element + mirror; then D = -2 tau on every row
                r0.add(sg, Wn);
                r0.add(tau, W[0]);
                rt.add(tau, Wt);
                rn = typename A::Acc();
            }
            if (minus || boundary) {              // D y enters with the edge's minus side (or its only side)
                r0.add(m2tau, sm.y[le][f][b]);
                rn.add(m2tau, sm.y[le][f][cn * P + b]);
                rt.add(m2tau, sm.y[le][f][ct * P + b]);
            }
            sm.h[le][f][b] = r0.get();
            sm.h[le][f][cn * P + b] = rn.get();
            sm.h[le][f][ct * P + b] = rt.get();
        }
    }
    __syncthreads();
    // boundary rows are complete; interior rows: leave this half (minus side in out, plus side in
    // half), then take the edge's ticket
    if (live) {
        for (int t = n; t < NFACE; t += Np) {
            const int f = t / NF, k = t % NF;
            const size_t o = (size_t)sm.ed[le][f] * NF + k;
            const TO v = (TO)A::to(sm.h[le][f][k]);
            if (sm.nb[le][f] < 0) {
                if constexpr (MODE == kMfResidual) out[o] = rhs[o] - v;
                else out[o] = v;
            } else if (f == 1 || f == 3) {
                out[o] = v;
            } else {
                half[o] = v;
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (live && n < 4)
        sm.second[le][n] = sm.nb[le][n] >= 0 ? atomicAdd(ticket + sm.ed[le][n], 1) : 0;
    __syncthreads();
    if (!live) return;
    __threadfence();
    for (int t = n; t < NFACE; t += Np) {
        const int f = t / NF, k = t % NF;
        if (sm.nb[le][f] < 0 || sm.second[le][f] != 1) continue;
        const size_t o = (size_t)sm.ed[le][f] * NF + k;
        const TO mine = (TO)A::to(sm.h[le][f][k]);
        const bool minus = f == 1 || f == 3;
        const TO sum = minus ? mine + __ldcg(half + o) : __ldcg(out + o) + mine;   // minus half first
        if constexpr (MODE == kMfResidual) out[o] = rhs[o] - sum;
        else out[o] = sum;
    }
    if (n < 4 && sm.nb[le][n] >= 0 && sm.second[le][n] == 1) ticket[sm.ed[le][n]] = 0;   // ready for the next product
}

// qhat = M^{-1} x~ with the FP32 block-Jacobi blocks, FP64-class sums (x split into FP32 pairs).
template <int NF>
__global__ void __launch_bounds__(256)
mf_back_kernel(int n_edges, const float* __restrict__ Minv, const double* __restrict__ x, double* __restrict__ y) {
    constexpr int EPB = 256 / NF;
    __shared__ float sxh[EPB][NF], sxl[EPB][NF];
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = blockIdx.x * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) split(x[(size_t)r * NF + ii], sxh[le][ii], sxl[le][ii]);
    __syncthreads();
    if (!live) return;
    const float* M = Minv + (size_t)r * NF * NF;
    Dot2 acc;
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) acc.add(M[jj * NF + ii], 0.f, sxh[le][jj], sxl[le][jj]);
    y[(size_t)r * NF + ii] = acc.value();
}

// hi parts of FP32 pairs
__global__ void pair_hi_kernel(const float2* __restrict__ a, float* __restrict__ hi, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        hi[t] = a[t].x;
}

template <int P, class A, int MODE, typename TX, typename TO>
cudaError_t mf_launch(const Geom& g, const void* S, const void* aux, const void* EG, const float* Minv,
                      const double* tau, const TX* x, const double* rhs, TO* out, void* half, int* ticket,
                      double beta, cudaStream_t s, const int* done) {
    using T = typename A::T;
    constexpr int EPB = mf_epb<P>();
    mf_trace_kernel<P, EPB, A, MODE><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(
        g, static_cast<const T*>(S), static_cast<const T*>(aux), static_cast<const T*>(EG), Minv, tau, x, rhs, out,
        reinterpret_cast<TO*>(half), ticket, beta, done);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mf_inner(const Geom& g, const MfOps& op, const float* x, float* y, double beta, cudaStream_t s,
                            const int* done) {
#define CASE(P)                                                                                               \
    case P:                                                                                                   \
        return mf_launch<P, ArithF32, kMfInner>(g, op.S32, op.aux32, op.EG32, op.Minv32, op.tau, x, nullptr, y, \
                                                op.half, op.ticket, beta, s, done);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_mf_residual(const Geom& g, const MfOps& op, const double* x, const double* rhs, double* w,
                               double beta, cudaStream_t s) {
#define CASE(P)                                                                                                \
    case P:                                                                                                    \
        return mf_launch<P, ArithF2, kMfResidual>(g, op.S2, op.aux2, op.EG2, op.Minv32, op.tau, x, rhs, w, op.half, \
                                                  op.ticket, beta, s, nullptr);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_mf_plain(const Geom& g, const MfOps& op, const double* x, double* y, double beta, cudaStream_t s) {
#define CASE(P)                                                                                                \
    case P:                                                                                                    \
        return mf_launch<P, ArithF2, kMfPlain>(g, op.S2, op.aux2, op.EG2, op.Minv32, op.tau, x, nullptr, y, op.half, \
                                               op.ticket, beta, s, nullptr);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_mf_back(const Geom& g, const float* Minv32, const double* x, double* y, cudaStream_t s) {
#define CASE(P, NF)                                                                                      \
    case P: {                                                                                            \
        constexpr int EPB = 256 / NF;                                                                    \
        mf_back_kernel<NF><<<(g.n_edges + EPB - 1) / EPB, EPB * NF, 0, s>>>(g.n_edges, Minv32, x, y);   \
        count_launches(1);                                                                               \
        return cudaGetLastError();                                                                       \
    }
    switch (g.P) {
        CASE(2, 6) CASE(3, 9) CASE(4, 12) CASE(5, 15) CASE(6, 18) CASE(7, 21) CASE(8, 24) CASE(9, 27)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_pair_hi(const void* pairs, float* hi, size_t n, cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pair_hi_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, 0, s>>>(static_cast<const float2*>(pairs), hi, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hdgdg
