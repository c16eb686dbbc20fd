// Element-local solves through the Schur complement on phi, shared by the local condensation /
// recovery kernels (kernels_hdg.cu) and the matrix-free trace operator (kernels_mf.cu).
//
// With collocated GLL nodes the velocity blocks of the element operator A are diagonal and equal
// to the phi block's diagonal d; eliminating U and V node by node leaves S phi = s with S the
// Schur complement, whose inverse is the (phi, phi) block of A^{-1} (block inversion).  The
// kernels keep per element that block, four numbers per node (1/d, -cx, -cy, phi_B) and two
// P x P coupling matrices per instance (-E, -G), and rebuild the rest.
#pragma once

#include "compensated.h"
#include "internal.h"

namespace hdgdg {

// Arithmetic of these solves.  ArithF64: FP64.  ArithF2: unevaluated FP32 pairs (hi, lo) with
// the compensated Dot2 sums of compensated.h -- FP64-class results on the FP32 pipes.
struct ArithF64 {
    using T = double;
    struct Acc {
        double s = 0.0;
        __device__ __forceinline__ void add(double a, double x) { s = fma(a, x, s); }
        __device__ __forceinline__ double get() const { return s; }
    };
    __device__ __forceinline__ static double from(double v) { return v; }
    __device__ __forceinline__ static double to(double v) { return v; }
    __device__ __forceinline__ static double mul(double a, double b) { return a * b; }
    // a small constant exact in FP32 (0, +-1, -2), at compile time
    __host__ __device__ static constexpr double cst(double v) { return v; }
};

struct ArithF2 {
    using T = float2;
    struct Acc {
        Dot2 d;
        __device__ __forceinline__ void add(float2 a, float2 x) { d.add(a.x, a.y, x.x, x.y); }
        __device__ __forceinline__ float2 get() const {
            float2 r;
            two_sum(d.p, d.c, r.x, r.y);
            return r;
        }
    };
    __device__ __forceinline__ static float2 from(double v) {
        float2 r;
        split(v, r.x, r.y);
        return r;
    }
    __device__ __forceinline__ static double to(float2 v) { return f32_to_f64(v.x) + f32_to_f64(v.y); }
    __host__ __device__ static constexpr float2 cst(double v) { return float2{(float)v, 0.f}; }
    // (a_hi + a_lo)(b_hi + b_lo): the exact a_hi b_hi (TwoProduct) plus the cross terms, renormalised
    __device__ __forceinline__ static float2 mul(float2 a, float2 b) {
        float p, e;
        two_prod(a.x, b.x, p, e);
        e = __fmaf_rn(a.x, b.y, e);
        e = __fmaf_rn(a.y, b.x, e);
        float2 r;
        r.x = __fadd_rn(p, e);
        r.y = __fsub_rn(e, __fsub_rn(r.x, p));
        return r;
    }
};

template <class A>
__device__ __forceinline__ void store_from(typename A::T* dst, double v) { *dst = A::from(v); }

// ArithF32: plain FP32 arithmetic (the inner cycles of the mixed form's trace solve).
struct ArithF32 {
    using T = float;
    struct Acc {
        float s = 0.f;
        __device__ __forceinline__ void add(float a, float x) { s = __fmaf_rn(a, x, s); }
        __device__ __forceinline__ float get() const { return s; }
    };
    __device__ __forceinline__ static float from(double v) { return f64_to_f32(v); }
    __device__ __forceinline__ static double to(float v) { return f32_to_f64(v); }
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __host__ __device__ static constexpr float cst(double v) { return (float)v; }
};

template <int P, int EPB, class A>
struct SchurSmem {
    using T = typename A::T;
    static constexpr int Np = P * P;
    T EG[EPB][2][Np];   // the element's -E, -G (P x P each, row major)
    T t[EPB][2][Np];    // d^{-1} x_U, d^{-1} x_V
    T s[EPB][Np];       // Schur right-hand side
    T w[EPB][Np];       // phi_B phi
};

// A load of operator data read once per pass, marked evict-first (ld.global.cs) so that it does
// not push out of L2 the vectors that the passes around it reuse.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
    return __ldcs(p);
}

// The four numbers per node the solve needs (1/d, -cx, -cy, phi_B), loaded at once (STREAM: as
// evict-first loads).
template <class A>
struct SchurNode {
    typename A::T rd{}, ncx{}, ncy{}, pb{};
    template <bool STREAM = false>
    __device__ __forceinline__ void load(const typename A::T* __restrict__ aux, int e, int n, int Np) {
        const typename A::T* ax = aux + (size_t)e * 4 * Np;
        if constexpr (STREAM) {
            rd = ld_stream(ax + n);
            ncx = ld_stream(ax + Np + n);
            ncy = ld_stream(ax + 2 * Np + n);
            pb = ld_stream(ax + 3 * Np + n);
        } else {
            rd = ax[n];
            ncx = ax[Np + n];
            ncy = ax[2 * Np + n];
            pb = ax[3 * Np + n];
        }
    }
};

// A^{-1} x for the element of thread (le, n) with x = (x0, xU, xV) at node n (each thread its
// own node's values); returns phi, U, V at node n.  Every thread of the block calls it (its
// barriers are block-wide); live marks threads of real elements.  nd holds the node's numbers;
// Srow(m) returns (S^{-1})_{n m}, the (phi, phi) block of A^{-1} (from memory or from registers
// the caller filled early).
template <int P, int EPB, class A, class SRow>
__device__ __forceinline__ void schur_solve_with(SchurSmem<P, EPB, A>& sm, const Geom& g, int e, int le, int n,
                                                 bool live, const SchurNode<A>& nd, SRow Srow,
                                                 const typename A::T* __restrict__ EG, typename A::T x0,
                                                 typename A::T xU, typename A::T xV, typename A::T& phi,
                                                 typename A::T& U, typename A::T& V) {
    using T = typename A::T;
    constexpr int Np = P * P;
    const int i = n % P, j = n / P;
    const T one = A::cst(1.0);
    if (live) {
        const T* eg = EG + (size_t)g.by_el.div(e) * 2 * Np;
        sm.EG[le][0][n] = eg[n];
        sm.EG[le][1][n] = eg[Np + n];
        sm.t[le][0][n] = A::mul(xU, nd.rd);
        sm.t[le][1][n] = A::mul(xV, nd.rd);
    }
    __syncthreads();
    if (live) {   // s = x_phi - Bx d^{-1} x_U - By d^{-1} x_V
        typename A::Acc acc;
        acc.add(one, x0);
#pragma unroll
        for (int a = 0; a < P; ++a) {
            acc.add(sm.EG[le][0][i * P + a], sm.t[le][0][j * P + a]);
            acc.add(sm.EG[le][0][j * P + a], sm.t[le][1][a * P + i]);
        }
        sm.s[le][n] = acc.get();
    }
    __syncthreads();
    if (live) {   // phi = S^{-1} s
        typename A::Acc acc;
#pragma unroll
        for (int m = 0; m < Np; ++m) acc.add(Srow(m), sm.s[le][m]);
        phi = acc.get();
        sm.w[le][n] = A::mul(nd.pb, phi);
    }
    __syncthreads();
    if (live) {   // d U = x_U - Cx phi,  d V = x_V - Cy phi
        typename A::Acc au, av;
        au.add(one, xU);
        au.add(nd.ncx, phi);
        av.add(one, xV);
        av.add(nd.ncy, phi);
#pragma unroll
        for (int a = 0; a < P; ++a) {
            au.add(sm.EG[le][1][i * P + a], sm.w[le][j * P + a]);
            av.add(sm.EG[le][1][j * P + a], sm.w[le][a * P + i]);
        }
        U = A::mul(au.get(), nd.rd);
        V = A::mul(av.get(), nd.rd);
    }
}

// The same with the node's numbers and S^{-1} read from memory (S [n_el][col m][row n]), as
// evict-first loads (each pass reads them once).
template <int P, int EPB, class A>
__device__ __forceinline__ void schur_solve(SchurSmem<P, EPB, A>& sm, const Geom& g, int e, int le, int n,
                                            bool live, const typename A::T* __restrict__ S,
                                            const typename A::T* __restrict__ aux,
                                            const typename A::T* __restrict__ EG, typename A::T x0,
                                            typename A::T xU, typename A::T xV, typename A::T& phi,
                                            typename A::T& U, typename A::T& V) {
    constexpr int Np = P * P;
    SchurNode<A> nd;
    if (live) nd.template load<true>(aux, e, n, Np);
    const typename A::T* Sn = S + (size_t)e * Np * Np + n;
    schur_solve_with<P, EPB, A>(sm, g, e, le, n, live, nd, [&](int m) { return ld_stream(Sn + (size_t)m * Np); },
                                EG, x0, xU, xV, phi, U, V);
}

}  // namespace hdgdg
