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
// Three launches per product in the refinement residual and the plain product, each short, so
// that no block waits on a chain of dependent memory round trips:
//   mf_pre_kernel   y = M^{-1} x, one thread per edge row (block-Jacobi inverse in scaled FP16);
//   mf_elem_kernel  one thread per (element, node): the node's traces y gathered straight into
//                   registers, the operator data loaded before them, the lift, the local solve,
//                   and the element's half of each face's row -- the edge's minus side (face 1 or
//                   3) into hm, its plus side into hp (a boundary face's full row into hm, 0 into hp);
//   mf_sum_kernel   y = hm + hp (residual mode: w = g - (hm + hp)), minus half first, so the
//                   result is the same whatever order the elements ran in.
// The inner cycles' product is ONE launch: the element pass first forms y = M^{-1} x on each face
// of its block's elements in shared memory (the same sums as mf_pre_kernel, term for term), and
// adds its half of each face's row into the output with a global reduction.  The output is zero
// beforehand and every row receives at most two addends, so the sum is the same in whichever order
// the two sides arrive (IEEE addition is commutative) and equals hm + hp of the three-pass form
// bit for bit -- apart from the sign of an exact zero, and halves below the FP32 normal range,
// which the reduction flushes to zero.
// Modes (the Krylov solve applies the block-Jacobi-preconditioned operator S~ = S M^{-1}):
//   kMfInner     y = S M^{-1} x        FP32 arithmetic and vectors (the mixed form's inner cycles)
//   kMfResidual  w = g - S M^{-1} x    FP64-class FP32-pair arithmetic, FP64 vectors (refinement)
//   kMfPlain     y = S x               FP64-class, FP64 vectors (the row-level entry point)
// M^{-1} is the block-Jacobi inverse held per edge as FP16 values of the block scaled by a power of
// two (PrecondBlocks); the inner cycles, the residual and the final back-transformation
// qhat = M^{-1} x~ use exactly these values, so the preconditioner is the same matrix on every path.
#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

#include "compensated.h"
#include "internal.h"
#include "schur.h"
#include "ens.h"

namespace hdgdg {
namespace {

enum MfMode { kMfInner = 0, kMfResidual = 1, kMfPlain = 2 };

template <int MODE>
using MfVec = std::conditional_t<MODE == kMfInner, float, double>;   // vectors of the mode

// Tiles of the element pass: elements per block for about `threads` threads (at most 32 elements),
// and whether the S^{-1} row is loaded into registers ahead of the traces.  Tile 0 is the default
// (256 threads, registers); the autotuner tries the others at create for degrees 2..4.
template <int P>
__host__ __device__ constexpr int mf_epb_for(int threads) {
    return threads / (P * P) > 32 ? 32 : (threads / (P * P) > 0 ? threads / (P * P) : 1);
}
template <int P>
__host__ __device__ constexpr int mf_epb() {
    return mf_epb_for<P>(256);
}
// tiles 6..8: no prefetch, registers capped for a full SM (64 warps) -- more elements in flight
constexpr int kMfTiles = 9;
constexpr int mf_tile_threads(int t) { return t % 3 == 0 ? 256 : t % 3 == 1 ? 128 : 512; }
constexpr bool mf_tile_pref(int t) { return t < 3; }
constexpr int mf_tile_minb(int t) { return t >= 6 ? 2048 / mf_tile_threads(t) : 1; }
// the refinement residual's FP32-pair pass holds ~112 registers a thread: its tiles 6..8 cap them
// at 85 (256 threads, 3 blocks an SM), 85 (128 threads, 6 blocks) and 64 (256 threads, 4 blocks)
constexpr int mf_res_threads(int t) { return t == 7 ? 128 : t >= 6 ? 256 : mf_tile_threads(t); }
constexpr int mf_res_minb(int t) { return t == 6 ? 3 : t == 7 ? 6 : t == 8 ? 4 : 1; }

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

// v * 2^k for an arithmetic value (exact: a power of two)
template <class A>
__device__ __forceinline__ typename A::T arith_scale(typename A::T v, float s) {
    if constexpr (std::is_same<typename A::T, float2>::value) return float2{v.x * s, v.y * s};
    else return v * (typename A::T)s;
}

// the element's half of a row, stored in the mode's vector type
template <class A, typename TO>
__device__ __forceinline__ TO arith_store(typename A::T v) {
    if constexpr (sizeof(typename A::T) == sizeof(float) && sizeof(TO) == sizeof(float)) return v;
    else return (TO)A::to(v);
}

// y = M^{-1} x per edge (one thread per row component), y in the arithmetic's own type
template <int NF, class A, typename TX>
__device__ __forceinline__ void mf_pre_body(int bid, int n_edges, PrecondBlocks Minv,
                                            const TX* __restrict__ x, typename A::T* __restrict__ y) {
    using T = typename A::T;
    constexpr int EPB = 256 / NF;
    __shared__ T xs[EPB][NF];
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = bid * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) xs[le][ii] = arith_load<A>(x + (size_t)r * NF + ii);
    __syncthreads();
    if (!live) return;
    const __half* M = Minv.h + (size_t)r * NF * NF + ii;
    typename A::Acc acc;
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) acc.add(arith_of_f32<A>(__half2float(M[jj * NF])), xs[le][jj]);
    y[(size_t)r * NF + ii] = arith_scale<A>(acc.get(), __ldg(Minv.scale + r));
}

template <int NF, class A, typename TX>
__global__ void __launch_bounds__(256)
mf_pre_kernel(int n_edges, PrecondBlocks Minv, const TX* __restrict__ x, typename A::T* __restrict__ y,
              const int* __restrict__ done) {
    if (done && *done) return;
    mf_pre_body<NF, A, TX>(blockIdx.x, n_edges, Minv, x, y);
}

// y = M^{-1} x on each face (slot le * 4 + f) of the block's elements, into ys -- the sums of
// mf_pre_body in the same order.  NF % 4 == 0: four rows per thread with 8-byte FP16 loads (x and
// M^{-1} 16- and 8-byte aligned, checked by the launcher); else one row per thread.
template <int P, int EPB>
__device__ __forceinline__ void mf_face_pre(int bid, const Geom& g, const PrecondBlocks& Minv,
                                            const float* __restrict__ x, float (*ys)[4][3 * P]) {
    constexpr int NF = 3 * P, NT = EPB * P * P;
    if constexpr (NF % 4 == 0) {
        constexpr int Q = NF / 4;
        for (int u = threadIdx.x; u < EPB * 4 * Q; u += NT) {
            const int slot = u / Q, q = u % Q, le = slot / 4, f = slot % 4;
            const int e = bid * EPB + le;
            if (e >= g.n_el) continue;
            const int r = edge_of_face(e, f, g);
            const float4* xr = reinterpret_cast<const float4*>(x + (size_t)r * NF);
            const __half* M = Minv.h + (size_t)r * NF * NF + 4 * q;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int jq = 0; jq < Q; ++jq) {
                const float4 xv = xr[jq];
                const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint2 mv = ld_stream(reinterpret_cast<const uint2*>(M + (size_t)(4 * jq + t) * NF));
                    const float2 m01 = __half22float2(*reinterpret_cast<const __half2*>(&mv.x));
                    const float2 m23 = __half22float2(*reinterpret_cast<const __half2*>(&mv.y));
                    a0 = __fmaf_rn(m01.x, xs[t], a0);
                    a1 = __fmaf_rn(m01.y, xs[t], a1);
                    a2 = __fmaf_rn(m23.x, xs[t], a2);
                    a3 = __fmaf_rn(m23.y, xs[t], a3);
                }
            }
            const float sc = __ldg(Minv.scale + r);
            ys[le][f][4 * q] = a0 * sc;
            ys[le][f][4 * q + 1] = a1 * sc;
            ys[le][f][4 * q + 2] = a2 * sc;
            ys[le][f][4 * q + 3] = a3 * sc;
        }
    } else {
        for (int u = threadIdx.x; u < EPB * 4 * NF; u += NT) {
            const int slot = u / NF, ii = u % NF, le = slot / 4, f = slot % 4;
            const int e = bid * EPB + le;
            if (e >= g.n_el) continue;
            const int r = edge_of_face(e, f, g);
            const float* xr = x + (size_t)r * NF;
            const __half* M = Minv.h + (size_t)r * NF * NF + ii;
            float a = 0.f;
#pragma unroll
            for (int jj = 0; jj < NF; ++jj) a = __fmaf_rn(__half2float(M[jj * NF]), xr[jj], a);
            ys[le][f][ii] = a * __ldg(Minv.scale + r);
        }
    }
}

// The element's half of each of its faces' rows at its node (see above): stored into hm / hp, or,
// FUSE, added into hm (the zeroed output).
template <int P, int EPB, class A, int MODE, bool FUSE>
__device__ __forceinline__ void mf_elem_rows(const Geom& g, int e, int le, const SchurNode<A>& nd, const bool* on,
                                             const int* fc, const int* bb, const int* ed,
                                             const typename A::T (*yv_)[3], const typename A::T* tau,
                                             typename A::T* W, double beta, MfVec<MODE>* __restrict__ hm,
                                             MfVec<MODE>* __restrict__ hp) {
    using T = typename A::T;
    using TO = MfVec<MODE>;
    constexpr int NF = 3 * P;
    const T bt = A::from(beta * dt_factor(g, e));
    W[0] = A::mul(bt, W[0]);
    W[1] = A::mul(bt, W[1]);
    W[2] = A::mul(bt, W[2]);
    const T one = A::cst(1.0), mone = A::cst(-1.0), mtwo = A::cst(-2.0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!on[k]) continue;
        const int f = fc[k], b = bb[k];
        const bool xedge = f < 2, minus = (f == 1 || f == 3);   // minus side: outward normal +axis
        const int cn = xedge ? 1 : 2, ct = xedge ? 2 : 1;
        const bool boundary = g.walls && neighbour(e, f, g) < 0;
        const size_t o = (size_t)ed[k] * NF + b;
        if (boundary && g.dirichlet) {   // prescribed trace: the identity row
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (FUSE) {
                    atomicAdd(hm + o + c * P, yv_[k][c]);
                } else {
                    hm[o + c * P] = arith_store<A, TO>(yv_[k][c]);
                    hp[o + c * P] = TO(0);
                }
            }
            continue;
        }
        const T Wn = W[cn], Wt = W[ct];
        const T sg = minus ? one : mone;
        const T m2tau = A::mul(mtwo, tau[k]);
        typename A::Acc r0, rn, rt;
        r0.add(sg, Wn);                       // U.n
        r0.add(tau[k], W[0]);                 // + tau phi
        rn.add(A::mul(sg, nd.pb), W[0]);      // phi_B phi n
        rn.add(tau[k], Wn);                   // + tau U_n
        rt.add(tau[k], Wt);                   // tau U_t
        if (boundary) {                       // wall: element + mirror; then D = -2 tau on every row
            r0.add(sg, Wn);
            r0.add(tau[k], W[0]);
            rt.add(tau[k], Wt);
            rn = typename A::Acc();
        }
        if (minus || boundary) {              // D y enters with the edge's minus side (or its only side)
            r0.add(m2tau, yv_[k][0]);
            rn.add(m2tau, yv_[k][cn]);
            rt.add(m2tau, yv_[k][ct]);
        }
        if constexpr (FUSE) {   // both sides into the zeroed output (a wall's one side is its whole row)
            atomicAdd(hm + o, r0.get());
            atomicAdd(hm + o + cn * P, rn.get());
            atomicAdd(hm + o + ct * P, rt.get());
            continue;
        }
        TO* dst = (minus || boundary) ? hm : hp;
        dst[o] = arith_store<A, TO>(r0.get());
        dst[o + cn * P] = arith_store<A, TO>(rn.get());
        dst[o + ct * P] = arith_store<A, TO>(rt.get());
        if (boundary) {
            hp[o] = TO(0);
            hp[o + cn * P] = TO(0);
            hp[o + ct * P] = TO(0);
        }
    }
}

// The element pass (see above).  PLAIN: y is the input vector itself (TX), else M^{-1} x (A::T).
// FUSE (inner mode): yv is x itself, y = M^{-1} x is formed per face in shared memory, and both
// halves of each row are added into hm (the zeroed output; hp unused).
// TAUN: tau_v holds tau_hat already in the arithmetic's type (FP32 for the fused pass, FP32 pairs
// for the refinement residual; converted once at setup), else in FP64.
template <int P, int EPB, class A, int MODE, bool PREF, bool FUSE = false, bool TAUN = FUSE>
__device__ __forceinline__ void mf_elem_body(int bid, const Geom& g, const typename A::T* __restrict__ S,
                                             const typename A::T* __restrict__ aux,
                                             const typename A::T* __restrict__ EG, const void* __restrict__ tau_v,
                                             const void* __restrict__ yv, MfVec<MODE>* __restrict__ hm,
                                             MfVec<MODE>* __restrict__ hp, double beta, PrecondBlocks Minv = {}) {
    using T = typename A::T;
    using TO = MfVec<MODE>;
    constexpr int Np = P * P, NF = 3 * P;
    constexpr bool kPref = PREF && Np <= 25;   // S^{-1} row loaded into registers ahead of the traces
    static_assert(!FUSE || (MODE == kMfInner && sizeof(T) == sizeof(float)), "the fused pass is the FP32 inner product");
    __shared__ SchurSmem<P, EPB, A> sm;
    __shared__ float ys[FUSE ? EPB : 1][4][FUSE ? NF : 1];
    const int le = threadIdx.x / Np, n = threadIdx.x % Np, i = n % P, j = n / P;
    const int e = bid * EPB + le;
    const bool live = le < EPB && e < g.n_el;
    // operator data first: it does not depend on the traces
    SchurNode<A> nd;
    T srow[kPref ? Np : 1];
    const T* Sn = S + (size_t)(live ? e : 0) * Np * Np + n;
    if (live) {
        nd.template load<true>(aux, e, n, Np);
        if constexpr (kPref) {
#pragma unroll
            for (int m = 0; m < Np; ++m) srow[m] = ld_stream(Sn + (size_t)m * Np);
        }
    }
    if constexpr (FUSE) {
        mf_face_pre<P, EPB>(bid, g, Minv, static_cast<const float*>(yv), ys);
        __syncthreads();
    }
    // the node's faces -- slot 0 its x-face (left or right), slot 1 its y-face (bottom or top) --
    // with the edge, the position along it, tau and the three trace components
    bool on[2];
    int fc[2], bb[2], ed[2] = {0, 0};
    on[0] = i == 0 || i == P - 1;
    fc[0] = i == 0 ? 0 : 1;
    bb[0] = j;
    on[1] = j == 0 || j == P - 1;
    fc[1] = j == 0 ? 2 : 3;
    bb[1] = i;
    T yv_[2][3];
    T tau[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        on[k] = on[k] && live;
        tau[k] = A::cst(0.0);
#pragma unroll
        for (int c = 0; c < 3; ++c) yv_[k][c] = A::cst(0.0);
        if (!on[k]) continue;
        const int r = edge_of_face(e, fc[k], g);
        ed[k] = r;
        if constexpr (TAUN) tau[k] = static_cast<const T*>(tau_v)[(size_t)r * P + bb[k]];
        else tau[k] = A::from(static_cast<const double*>(tau_v)[(size_t)r * P + bb[k]]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = (size_t)r * NF + c * P + bb[k];
            if constexpr (FUSE) yv_[k][c] = ys[le][fc[k]][c * P + bb[k]];
            else if constexpr (MODE == kMfPlain) yv_[k][c] = A::from(static_cast<const double*>(yv)[o]);
            else yv_[k][c] = static_cast<const T*>(yv)[o];
        }
    }
    // lift: u = sum over the node's faces of tau y
    T u[3];
    {
        typename A::Acc a0, a1, a2;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!on[k]) continue;
            a0.add(tau[k], yv_[k][0]);
            a1.add(tau[k], yv_[k][1]);
            a2.add(tau[k], yv_[k][2]);
        }
        u[0] = a0.get();
        u[1] = a1.get();
        u[2] = a2.get();
    }
    T W[3];
    if constexpr (kPref)
        schur_solve_with<P, EPB, A>(sm, g, e, le, n, live, nd, [&](int m) { return srow[m]; }, EG, u[0], u[1],
                                    u[2], W[0], W[1], W[2]);
    else
        schur_solve_with<P, EPB, A>(sm, g, e, le, n, live, nd, [&](int m) { return ld_stream(Sn + (size_t)m * Np); },
                                    EG, u[0], u[1], u[2], W[0], W[1], W[2]);
    if (live) mf_elem_rows<P, EPB, A, MODE, FUSE>(g, e, le, nd, on, fc, bb, ed, yv_, tau, W, beta, hm, hp);
}

template <int P, int EPB, class A, int MODE, bool PREF, int MINB = 1, bool FUSE = false, bool TAUN = FUSE>
__global__ void __launch_bounds__(EPB * P * P, MINB)
    mf_elem_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                   const typename A::T* __restrict__ EG, const void* __restrict__ tau_edge,
                   const void* __restrict__ yv, MfVec<MODE>* __restrict__ hm, MfVec<MODE>* __restrict__ hp,
                   double beta, PrecondBlocks Minv, const int* __restrict__ done) {
    if (done && *done) return;
    mf_elem_body<P, EPB, A, MODE, PREF, FUSE, TAUN>(blockIdx.x, g, S, aux, EG, tau_edge, yv, hm, hp, beta, Minv);
}

// y = 0 (the fused product's output, when the caller has not zeroed it)
__global__ void __launch_bounds__(256) zero_f32_kernel(float* __restrict__ y, size_t n, const int* __restrict__ done) {
    if (done && *done) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        y[t] = 0.f;
}


// y = hm + hp, or w = g - (hm + hp)
template <typename TO, bool RESID>
__global__ void __launch_bounds__(256)
mf_sum_kernel(size_t n, const TO* __restrict__ hm, const TO* __restrict__ hp, const double* __restrict__ rhs,
              TO* __restrict__ out, const int* __restrict__ done) {
    if (done && *done) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const TO v = hm[t] + hp[t];
        if constexpr (RESID) out[t] = rhs[t] - v;
        else out[t] = v;
    }
}

// qhat = M^{-1} x~ with the FP32 block-Jacobi blocks, FP64-class sums (x split into FP32 pairs).
template <int NF>
__device__ __forceinline__ void mf_back_body(int bid, int n_edges, PrecondBlocks Minv,
                                             const double* __restrict__ x, double* __restrict__ y) {
    constexpr int EPB = 256 / NF;
    __shared__ float sxh[EPB][NF], sxl[EPB][NF];
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = bid * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) split(x[(size_t)r * NF + ii], sxh[le][ii], sxl[le][ii]);
    __syncthreads();
    if (!live) return;
    const __half* M = Minv.h + (size_t)r * NF * NF;
    Dot2 acc;
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) acc.add(__half2float(M[jj * NF + ii]), 0.f, sxh[le][jj], sxl[le][jj]);
    const float sc = Minv.scale[r];   // a power of two: scaling the pair is exact
    y[(size_t)r * NF + ii] = f32_to_f64(acc.p * sc) + f32_to_f64(acc.c * sc);
}

template <int NF>
__global__ void __launch_bounds__(256)
mf_back_kernel(int n_edges, PrecondBlocks Minv, const double* __restrict__ x, double* __restrict__ y) {
    mf_back_body<NF>(blockIdx.x, n_edges, Minv, x, y);
}

// The two FP64-class block-Jacobi products -- the refinement residual's y = M^{-1} x as FP32 pairs
// (PAIRS) and the back-transformation qhat = M^{-1} x~ in FP64 -- with four rows per thread
// (NF % 4 == 0): the edge's x split into FP32 pairs in shared memory by its threads, then four
// Dot2 sums over the edge's NF columns from 8-byte FP16 loads.  Each row's sum is mf_pre_body's
// (ArithF2) or mf_back_body's, term for term.
template <int NF, bool PAIRS>
__global__ void __launch_bounds__(256)
    mf_edge_quad_kernel(int n_edges, PrecondBlocks Minv, const double* __restrict__ x, void* __restrict__ yv) {
    static_assert(NF % 4 == 0, "four rows per thread");
    constexpr int Q = NF / 4, EPB = 256 / Q;
    __shared__ float sxh[EPB][NF], sxl[EPB][NF];
    const int le = threadIdx.x / Q, q = threadIdx.x % Q;
    const int r = blockIdx.x * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) {
#pragma unroll
        for (int t = 0; t < 4; ++t) split(x[(size_t)r * NF + 4 * q + t], sxh[le][4 * q + t], sxl[le][4 * q + t]);
    }
    __syncthreads();
    if (!live) return;
    const __half* M = Minv.h + (size_t)r * NF * NF + 4 * q;
    Dot2 acc[4];
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) {
        const uint2 mv = ld_stream(reinterpret_cast<const uint2*>(M + jj * NF));
        const float2 m01 = __half22float2(*reinterpret_cast<const __half2*>(&mv.x));
        const float2 m23 = __half22float2(*reinterpret_cast<const __half2*>(&mv.y));
        const float xh = sxh[le][jj], xl = sxl[le][jj];
        acc[0].add(m01.x, 0.f, xh, xl);
        acc[1].add(m01.y, 0.f, xh, xl);
        acc[2].add(m23.x, 0.f, xh, xl);
        acc[3].add(m23.y, 0.f, xh, xl);
    }
    const float sc = Minv.scale[r];   // a power of two: scaling the pair is exact
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const size_t o = (size_t)r * NF + 4 * q + t;
        if constexpr (PAIRS) {
            float2 pr;
            two_sum(acc[t].p, acc[t].c, pr.x, pr.y);
            static_cast<float2*>(yv)[o] = float2{pr.x * sc, pr.y * sc};
        } else {
            static_cast<double*>(yv)[o] = f32_to_f64(acc[t].p * sc) + f32_to_f64(acc[t].c * sc);
        }
    }
}

template <int NF, bool PAIRS>
void mf_edge_quad_launch(int n_edges, const PrecondBlocks& Minv, const double* x, void* y, cudaStream_t s) {
    constexpr int EPB = 256 / (NF / 4);
    mf_edge_quad_kernel<NF, PAIRS><<<(n_edges + EPB - 1) / EPB, EPB * (NF / 4), 0, s>>>(n_edges, Minv, x, y);
}

// Setup: per edge (one block) the FP16 block-Jacobi inverse scaled by the power of two 2^e with
// max |entry| / 2^e in [0.5, 1), and that scale.
__global__ void precond_f16_kernel(const double* __restrict__ Minv, int NF, __half* __restrict__ h,
                                   float* __restrict__ scale) {
    const int r = blockIdx.x;
    const double* M = Minv + (size_t)r * NF * NF;
    __shared__ double red[256];
    double m = 0.0;
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) m = fmax(m, fabs(M[t]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    int e = 0;
    (void)frexp(red[0], &e);
    if (red[0] == 0.0) e = 0;
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) h[(size_t)r * NF * NF + t] = __double2half(ldexp(M[t], -e));
    if (threadIdx.x == 0) scale[r] = ldexpf(1.0f, e);
}

// hi parts of FP32 pairs
__global__ void pair_hi_kernel(const float2* __restrict__ a, float* __restrict__ hi, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        hi[t] = a[t].x;
}

int sum_grid(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b > 0 ? (int)b : 1;
}

template <int P, class A, int MODE, int TILE>
void mf_elem_launch(const Geom& g, const void* S, const void* aux, const void* EG, const void* tau, const void* yv,
                    MfVec<MODE>* hm, MfVec<MODE>* hp, double beta, cudaStream_t s, const int* done,
                    const PrecondBlocks& Minv) {
    using T = typename A::T;
    constexpr bool kRes = MODE == kMfResidual;
    constexpr int EPB = mf_epb_for<P>(kRes ? mf_res_threads(TILE) : mf_tile_threads(TILE));
    constexpr int kMinB = kRes ? mf_res_minb(TILE) : mf_tile_minb(TILE);
    constexpr bool kFuse = MODE == kMfInner;
    constexpr bool kTauN = MODE != kMfPlain;   // the inner and residual modes read their own copy of tau
    mf_elem_kernel<P, EPB, A, MODE, mf_tile_pref(TILE), kMinB, kFuse, kTauN>
        <<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(g, static_cast<const T*>(S), static_cast<const T*>(aux),
                                                          static_cast<const T*>(EG), tau, yv, hm, hp, beta, Minv,
                                                          done);
}

// the element pass with tile t (degrees 2..4: tiles 0..8 in the inner cycles and in the
// refinement residual; tile 0 elsewhere)
template <int P, class A, int MODE>
void mf_elem_tile(int t, const Geom& g, const void* S, const void* aux, const void* EG, const void* tau,
                  const void* yv, MfVec<MODE>* hm, MfVec<MODE>* hp, double beta, cudaStream_t s, const int* done,
                  const PrecondBlocks& Minv) {
    if constexpr (MODE == kMfResidual && P >= 3 && P <= 5) {
        switch (t) {
            case 1: return mf_elem_launch<P, A, MODE, 1>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 2: return mf_elem_launch<P, A, MODE, 2>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 3: return mf_elem_launch<P, A, MODE, 3>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 4: return mf_elem_launch<P, A, MODE, 4>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 5: return mf_elem_launch<P, A, MODE, 5>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 6: return mf_elem_launch<P, A, MODE, 6>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 7: return mf_elem_launch<P, A, MODE, 7>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 8: return mf_elem_launch<P, A, MODE, 8>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            default: break;
        }
    }
    if constexpr (MODE == kMfInner && P >= 3 && P <= 5) {
        switch (t) {
            case 1: return mf_elem_launch<P, A, MODE, 1>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 2: return mf_elem_launch<P, A, MODE, 2>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 3: return mf_elem_launch<P, A, MODE, 3>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 4: return mf_elem_launch<P, A, MODE, 4>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 5: return mf_elem_launch<P, A, MODE, 5>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 6: return mf_elem_launch<P, A, MODE, 6>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 7: return mf_elem_launch<P, A, MODE, 7>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            case 8: return mf_elem_launch<P, A, MODE, 8>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
            default: break;
        }
    }
    mf_elem_launch<P, A, MODE, 0>(g, S, aux, EG, tau, yv, hm, hp, beta, s, done, Minv);
}

// One product: [y = M^{-1} x,] the element pass, the edge sum; the inner mode's fused pass alone
// (after zeroing the output unless out_zeroed).
template <int P, class A, int MODE>
cudaError_t mf_launch(const Geom& g, const MfOps& op, const void* S, const void* aux, const void* EG, const void* x,
                      const double* rhs, MfVec<MODE>* out, double beta, cudaStream_t s, const int* done,
                      bool out_zeroed = false, double* nrm_scratch = nullptr, double* nrm_out = nullptr) {
    using T = typename A::T;
    using TO = MfVec<MODE>;
    constexpr int NF = 3 * P;
    if constexpr (MODE == kMfInner) {
        // the fused pass's vector loads (NF % 4 == 0): x on 16 bytes, the FP16 blocks on 8
        if (NF % 4 == 0 &&
            (reinterpret_cast<uintptr_t>(x) % 16 != 0 || reinterpret_cast<uintptr_t>(op.Minv.h) % 8 != 0))
            return cudaErrorMisalignedAddress;
        const size_t n = (size_t)g.n_edges * NF;
        if (!out_zeroed) {
            zero_f32_kernel<<<sum_grid(n), 256, 0, s>>>(reinterpret_cast<float*>(out), n, done);
            count_launches(1);
        }
        if (!op.tau32) return cudaErrorInvalidValue;   // the fused pass reads the FP32 copy of tau
        mf_elem_tile<P, A, MODE>(op.tile, g, S, aux, EG, op.tau32, x, out, nullptr, beta, s, done, op.Minv);
        count_launches(1);
        return cudaGetLastError();
    }
    const void* yv = x;
    if constexpr (MODE != kMfPlain) {
        if constexpr (MODE == kMfResidual && NF % 4 == 0) {
            mf_edge_quad_launch<NF, true>(g.n_edges, op.Minv, static_cast<const double*>(x), op.ybuf, s);
        } else {
            constexpr int EPE = 256 / NF;
            mf_pre_kernel<NF, A, TO><<<(g.n_edges + EPE - 1) / EPE, EPE * NF, 0, s>>>(
                g.n_edges, op.Minv, static_cast<const TO*>(x), static_cast<T*>(op.ybuf), done);
        }
        yv = op.ybuf;
    }
    TO* hm = static_cast<TO*>(op.hm);
    TO* hp = static_cast<TO*>(op.hp);
    if (MODE == kMfResidual && !op.tau2) return cudaErrorInvalidValue;
    mf_elem_tile<P, A, MODE>(MODE == kMfResidual ? op.tile_res : 0, g, S, aux, EG,
                             MODE == kMfResidual ? op.tau2 : static_cast<const void*>(op.tau), yv, hm, hp, beta, s,
                             done, op.Minv);
    const size_t n = (size_t)g.n_edges * NF;
    if constexpr (MODE == kMfResidual) {
        if (nrm_scratch) {   // the last pass with ||w||^2
            count_launches(2);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            return launch_sum_residual_norm(n, hm, hp, rhs, out, nrm_scratch, nrm_out, s);
        }
    }
    mf_sum_kernel<TO, MODE == kMfResidual><<<sum_grid(n), 256, 0, s>>>(n, hm, hp, rhs, out, done);
    count_launches(MODE != kMfPlain ? 3 : 2);
    return cudaGetLastError();
}

// ---- ensembles: the operator's three passes over every group, one persistent launch each -----------
template <class A, typename TX>
__global__ void __launch_bounds__(256) ens_mf_pre_kernel(EnsTable t, const TX* __restrict__ x,
                                                         typename A::T* __restrict__ y, const int* __restrict__ done) {
    if (done && *done) return;
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        switch (G.g.P) {
            case 3: mf_pre_body<9, A, TX>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            case 4: mf_pre_body<12, A, TX>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            case 5: mf_pre_body<15, A, TX>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            default: break;
        }
    });
}

template <class A, int MODE>
__global__ void __launch_bounds__(256) ens_mf_elem_kernel(EnsTable t, const typename A::T* __restrict__ y,
                                                          MfVec<MODE>* __restrict__ hm, MfVec<MODE>* __restrict__ hp,
                                                          const int* __restrict__ done) {
    if (done && *done) return;
    constexpr bool k32 = sizeof(typename A::T) == sizeof(float);
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        using T = typename A::T;
        const T* S = k32 ? reinterpret_cast<const T*>(G.S32) : static_cast<const T*>(G.S2);
        const T* aux = k32 ? reinterpret_cast<const T*>(G.aux32) : static_cast<const T*>(G.aux2);
        const T* EG = k32 ? reinterpret_cast<const T*>(G.EG32) : static_cast<const T*>(G.EG2);
        const size_t o = G.offt;
        switch (G.g.P) {
            case 3: mf_elem_body<3, mf_epb<3>(), A, MODE, true>(bid, G.g, S, aux, EG, G.tau, y + o, hm + o, hp + o, G.beta); break;
            case 4: mf_elem_body<4, mf_epb<4>(), A, MODE, true>(bid, G.g, S, aux, EG, G.tau, y + o, hm + o, hp + o, G.beta); break;
            case 5: mf_elem_body<5, mf_epb<5>(), A, MODE, true>(bid, G.g, S, aux, EG, G.tau, y + o, hm + o, hp + o, G.beta); break;
            default: break;
        }
    });
}

__global__ void __launch_bounds__(256) ens_mf_back_kernel(EnsTable t, const double* __restrict__ x, double* __restrict__ y) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        switch (G.g.P) {
            case 3: mf_back_body<9>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            case 4: mf_back_body<12>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            case 5: mf_back_body<15>(bid, G.g.n_edges, G.Minv, x + G.offt, y + G.offt); break;
            default: break;
        }
    });
}

int ens_edge_blocks(const EnsGroup& G) {
    const int epb = 256 / (3 * G.g.P);
    return (G.g.n_edges + epb - 1) / epb;
}

int ens_mf_elem_blocks(const EnsGroup& G) {
    const int P = G.g.P, epb = 256 / (P * P) > 32 ? 32 : 256 / (P * P);
    return (G.g.n_el + epb - 1) / epb;
}

template <class A, int MODE>
cudaError_t ens_mf_launch(const EnsHost& E, const MfOps& op, size_t nt, const MfVec<MODE>* x, const double* rhs,
                          MfVec<MODE>* out, cudaStream_t s, const int* done) {
    using T = typename A::T;
    using TO = MfVec<MODE>;
    const EnsTable te = ens_table(E, ens_edge_blocks);
    const EnsTable tm = ens_table(E, ens_mf_elem_blocks);
    T* y = static_cast<T*>(op.ybuf);
    TO* hm = static_cast<TO*>(op.hm);
    TO* hp = static_cast<TO*>(op.hp);
    ens_mf_pre_kernel<A, TO><<<ens_grid(ens_mf_pre_kernel<A, TO>, te.start[te.ngroups]), 256, 0, s>>>(te, x, y, done);
    ens_mf_elem_kernel<A, MODE><<<ens_grid(ens_mf_elem_kernel<A, MODE>, tm.start[tm.ngroups]), 256, 0, s>>>(tm, y, hm,
                                                                                                         hp, done);
    mf_sum_kernel<TO, MODE == kMfResidual><<<sum_grid(nt), 256, 0, s>>>(nt, hm, hp, rhs, out, done);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mf_inner(const Geom& g, const MfOps& op, const float* x, float* y, double beta, cudaStream_t s,
                            const int* done, bool y_zeroed) {
#define CASE(P)                                                                                                 \
    case P:                                                                                                     \
        return mf_launch<P, ArithF32, kMfInner>(g, op, op.S32, op.aux32, op.EG32, x, nullptr, y, beta, s, done, \
                                                y_zeroed);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_mf_residual(const Geom& g, const MfOps& op, const double* x, const double* rhs, double* w,
                               double beta, cudaStream_t s, double* nrm_scratch, double* nrm_out) {
#define CASE(P)                                                                                                 \
    case P:                                                                                                     \
        return mf_launch<P, ArithF2, kMfResidual>(g, op, op.S2, op.aux2, op.EG2, x, rhs, w, beta, s, nullptr, \
                                                  false, nrm_scratch, nrm_out);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_mf_plain(const Geom& g, const MfOps& op, const double* x, double* y, double beta, cudaStream_t s) {
#define CASE(P) \
    case P: return mf_launch<P, ArithF2, kMfPlain>(g, op, op.S2, op.aux2, op.EG2, x, nullptr, y, beta, s, nullptr);
    switch (g.P) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

// Time each tile of the inner cycles' element pass on the handle's own operators (two warm-up and
// five timed products each, CUDA events on the stream; x and y are scratch trace vectors) and keep
// the fastest in op.tile; then the refinement residual's tiles (xd, rhs, w: scratch FP64 trace
// vectors) into op.tile_res.  The tile changes no thread's arithmetic, only how elements share blocks.
cudaError_t launch_mf_autotune(const Geom& g, MfOps& op, const float* x, float* y, const double* xd,
                               const double* rhs, double* w, double beta, cudaStream_t s, int* epb, int* prefetch) {
    op.tile = 0;
    op.tile_res = 0;
    *epb = 0;
    *prefetch = 0;
    if (g.P < 3 || g.P > 5) return cudaSuccess;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return cudaGetLastError();
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return cudaGetLastError();
    }
    float best = 1e30f;
    int best_t = 0;
    cudaError_t err = cudaSuccess;
    for (int t = 0; t < kMfTiles && err == cudaSuccess; ++t) {
        op.tile = t;
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) err = launch_mf_inner(g, op, x, y, beta, s);
        if (err == cudaSuccess) err = cudaEventRecord(a, s);
        for (int k = 0; k < 5 && err == cudaSuccess; ++k) err = launch_mf_inner(g, op, x, y, beta, s);
        if (err == cudaSuccess) err = cudaEventRecord(b, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            best_t = t;
        }
    }
    op.tile = best_t;
    // the refinement residual's element pass (FP32 pairs): tiles 0..8 (6..8 with capped registers)
    best = 1e30f;
    int best_r = 0;
    for (int t = 0; t < kMfTiles && err == cudaSuccess; ++t) {
        op.tile_res = t;
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) err = launch_mf_residual(g, op, xd, rhs, w, beta, s);
        if (err == cudaSuccess) err = cudaEventRecord(a, s);
        for (int k = 0; k < 5 && err == cudaSuccess; ++k) err = launch_mf_residual(g, op, xd, rhs, w, beta, s);
        if (err == cudaSuccess) err = cudaEventRecord(b, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            best_r = t;
        }
    }
    op.tile_res = best_r;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    mf_tile_info(g.P, best_t, epb, prefetch);
    return err;
}

bool mf_tile_ready(int P, int t) { return t == 0 || (P >= 3 && P <= 5 && t > 0 && t < kMfTiles); }

void mf_tile_info(int P, int t, int* epb, int* prefetch) {
    const int th = mf_tile_threads(t);
    *epb = th / (P * P) > 32 ? 32 : (th / (P * P) > 0 ? th / (P * P) : 1);
    *prefetch = mf_tile_pref(t) ? 1 : 0;
}

cudaError_t launch_ens_mf_inner(const EnsHost& E, const MfOps& scratch, size_t nt, const float* x, float* y,
                                cudaStream_t s, const int* done) {
    return ens_mf_launch<ArithF32, kMfInner>(E, scratch, nt, x, nullptr, y, s, done);
}

cudaError_t launch_ens_mf_residual(const EnsHost& E, const MfOps& scratch, size_t nt, const double* x,
                                   const double* rhs, double* w, cudaStream_t s) {
    return ens_mf_launch<ArithF2, kMfResidual>(E, scratch, nt, x, rhs, w, s, nullptr);
}

cudaError_t launch_ens_mf_back(const EnsHost& E, const double* x, double* y, cudaStream_t s) {
    const EnsTable te = ens_table(E, ens_edge_blocks);
    ens_mf_back_kernel<<<ens_grid(ens_mf_back_kernel, te.start[te.ngroups]), 256, 0, s>>>(te, x, y);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mf_back(const Geom& g, const PrecondBlocks& Minv, const double* x, double* y, cudaStream_t s) {
#define CASE(P, NF)                                                                                      \
    case P: {                                                                                            \
        constexpr int EPB = 256 / NF;                                                                    \
        if constexpr (NF % 4 == 0) mf_edge_quad_launch<NF, false>(g.n_edges, Minv, x, y, s);             \
        else mf_back_kernel<NF><<<(g.n_edges + EPB - 1) / EPB, EPB * NF, 0, s>>>(g.n_edges, Minv, x, y); \
        count_launches(1);                                                                               \
        return cudaGetLastError();                                                                       \
    }
    switch (g.P) {
        CASE(2, 6) CASE(3, 9) CASE(4, 12) CASE(5, 15) CASE(6, 18) CASE(7, 21) CASE(8, 24) CASE(9, 27)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

cudaError_t launch_precond_f16(const double* Minv, int n_edges, int NF, __half* h, float* scale, cudaStream_t s) {
    precond_f16_kernel<<<n_edges, 256, 0, s>>>(Minv, NF, h, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_hi(const void* pairs, float* hi, size_t n, cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pair_hi_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, 0, s>>>(static_cast<const float2*>(pairs), hi, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hdgdg
