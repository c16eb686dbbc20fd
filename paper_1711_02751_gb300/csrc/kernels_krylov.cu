// Krylov kernel set for the condensed trace system (Sec. 6, eq. linearizedHDGsystem_schur).
//
// The paper factorises the trace matrix once with a sparse direct LU; here the system is
// solved by right-preconditioned GMRES(m) with classical Gram-Schmidt applied twice.  The
// block-Jacobi preconditioner (inverse of each edge's diagonal n_f x n_f block) is folded
// into the stored matrix once at setup, S~ = S M^{-1}, so the diagonal blocks of S~ are the
// identity and are not stored.  All reductions use a fixed grid and a fixed summation
// order, so results are bitwise reproducible run to run.
//
// Every kernel is a template on the storage type T: double for the FP64 path, float for the
// inner solves of the mixed-precision path.  Products and per-thread partial sums are in T;
// warp, block and grid reductions are in double.  The trace-matrix products are in
// kernels_spmv.cu.
#include <cstdint>
#include <initializer_list>

#include "compensated.h"
#include "internal.h"
#include "reduce.h"

namespace hdgdg {
namespace {

constexpr int kDotBlocks = 608;    // 4 x 152 SMs
constexpr int kDotThreads = 256;
constexpr int kDotChunk = 8;       // vectors reduced per pass over w

// VW consecutive entries of a vector: one 16-byte load or store for VW = 4 (FP32), one entry for
// VW = 1.  Index i counts groups of VW entries; the launchers use VW = 4 only when every vector
// involved starts on a 16-byte boundary and n is a multiple of 4.
template <typename T, int VW>
struct Lanes {
    T v[VW];
};

template <typename T, int VW>
__device__ __forceinline__ Lanes<T, VW> load_lanes(const T* __restrict__ p, size_t i) {
    Lanes<T, VW> r;
    if constexpr (VW == 4) {
        const float4 q = reinterpret_cast<const float4*>(p)[i];
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    } else if constexpr (VW == 2) {
        static_assert(sizeof(T) == 8, "16-byte lanes of FP64");
        const double2 q = reinterpret_cast<const double2*>(p)[i];
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        r.v[0] = p[i];
    }
    return r;
}

template <typename T, int VW>
__device__ __forceinline__ void store_lanes(T* __restrict__ p, size_t i, const Lanes<T, VW>& r) {
    if constexpr (VW == 4) reinterpret_cast<float4*>(p)[i] = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    else if constexpr (VW == 2) reinterpret_cast<double2*>(p)[i] = make_double2(r.v[0], r.v[1]);
    else p[i] = r.v[0];
}

// y[r] = B_r x[r] for column-major NF x NF blocks (FP64)
template <int NF>
__global__ void __launch_bounds__(256)
block_diag_kernel(int n_edges, const double* __restrict__ Bd, const double* __restrict__ x,
                  double* __restrict__ y) {
    constexpr int EPB = 256 / NF;
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = blockIdx.x * EPB + le;
    if (le >= EPB || r >= n_edges) return;
    const double* B = Bd + (size_t)r * NF * NF;
    const double* xr = x + (size_t)r * NF;
    double acc = 0.0;
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) acc += B[jj * NF + ii] * xr[jj];
    y[(size_t)r * NF + ii] = acc;
}

// The same product with the blocks held as FP32 pairs (float2 (hi, lo), in place of the FP64
// blocks) and compensated Dot2 sums (compensated.h); each x entry is split once, into shared memory.
template <int NF>
__global__ void __launch_bounds__(256)
block_diag_x2_kernel(int n_edges, const float2* __restrict__ Bd, const double* __restrict__ x,
                     double* __restrict__ y) {
    constexpr int EPB = 256 / NF;
    __shared__ float sxh[EPB][NF], sxl[EPB][NF];
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = blockIdx.x * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) split(x[(size_t)r * NF + ii], sxh[le][ii], sxl[le][ii]);
    __syncthreads();
    if (!live) return;
    const float2* B = Bd + (size_t)r * NF * NF;
    Dot2 acc;
#pragma unroll
    for (int jj = 0; jj < NF; ++jj) {
        const float2 bv = B[jj * NF + ii];
        acc.add(bv.x, bv.y, sxh[le][jj], sxl[le][jj]);
    }
    y[(size_t)r * NF + ii] = acc.value();
}

// a[i] (FP64) -> its FP32 pair (hi, lo) stored in the same eight bytes
__global__ void split_pairs_inplace_kernel(double* a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 pr;
        split(a[i], pr.x, pr.y);
        reinterpret_cast<float2*>(a)[i] = pr;
    }
}

__device__ void gmres_arnoldi_update(GmresCtl* c, int j, int m, const double* h1, const double* h2,
                                     const double* hn);

// out[j0 + c] = V_{j0+c} . w, c < nj: block partials in scratch, summed by the last block
template <int CH, typename T, int VW = 1>
__global__ void __launch_bounds__(kDotThreads)
multidot_kernel(const T* __restrict__ V, size_t ldv, int j0, int nj, const T* __restrict__ w,
                size_t n, double* __restrict__ scratch, int ldp, double* __restrict__ out,
                const int* __restrict__ done) {
    if (done && *done) return;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[CH][kDotThreads / 32];
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = T(0);
    for (size_t iv = blockIdx.x * (size_t)kDotThreads + threadIdx.x; iv < n / VW;
         iv += (size_t)gridDim.x * kDotThreads) {
        const Lanes<T, VW> wv = load_lanes<T, VW>(w, iv);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (c < nj) {
                const Lanes<T, VW> v = load_lanes<T, VW>(V + (size_t)(j0 + c) * ldv, iv);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[c] += v.v[k] * wv.v[k];
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const double s = warp_sum((double)acc[c]);
        if (lane == 0) sh[c][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < CH && (int)threadIdx.x < nj) {
        double s = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) s += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * ldp + j0 + threadIdx.x] = s;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, ldp, j0, nj, out + j0);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// v = w / sqrt(*nrm2) (w in FP64, v in T); zero[idx] = 0 when given
template <typename T>
__global__ void scale_kernel(const double* __restrict__ w, const double* __restrict__ nrm2,
                             T* __restrict__ v, size_t n, T* __restrict__ zero) {
    const double s = 1.0 / sqrt(*nrm2);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        v[idx] = from_f64<T>(w[idx] * s);
        if (zero) zero[idx] = T(0);
    }
}

__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x)
        b[idx] = (float)a[idx];
}

// Second Gram-Schmidt pass fused with the update of the first: w1 = w - sum_j h1_j V_j (w
// overwritten), and V_j . w1 (j < NJ) -> h2 and w1 . w1 -> nw1, the V_j kept in registers.  The
// last block also forms hn = sqrt(||w1||^2 - ||h2||^2), the norm of w2 = w1 - V h2 for an
// orthonormal V, and, given a GMRES control block, the Hessenberg column j with its Givens
// rotation and stop test.
// TWICE = false (classical Gram-Schmidt once): only the update and ||w1||; h2 = 0, hn = ||w1||.
template <int NJ, typename T, bool TWICE, int VW = 1>
__global__ void __launch_bounds__(kDotThreads)
axpy_dot_kernel(const T* __restrict__ V, size_t ldv, const double* __restrict__ h1, T* __restrict__ w,
                size_t n, double* __restrict__ scratch, double* __restrict__ h2, double* __restrict__ nw1,
                double* __restrict__ hn, GmresCtl* ctl, int jcol, int m, const int* __restrict__ done) {
    if (done && *done) return;
    constexpr int ldp = NJ + 1;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[NJ + 1][kDotThreads / 32];
    T hc[NJ], acc[NJ + 1];
#pragma unroll
    for (int j = 0; j < NJ; ++j) { hc[j] = T(__ldg(h1 + j)); acc[j] = T(0); }
    acc[NJ] = T(0);
    for (size_t iv = blockIdx.x * (size_t)kDotThreads + threadIdx.x; iv < n / VW;
         iv += (size_t)gridDim.x * kDotThreads) {
        Lanes<T, VW> v[NJ];
        Lanes<T, VW> x = load_lanes<T, VW>(w, iv);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            v[j] = load_lanes<T, VW>(V + (size_t)j * ldv, iv);
#pragma unroll
            for (int k = 0; k < VW; ++k) x.v[k] -= hc[j] * v[j].v[k];
        }
        store_lanes<T, VW>(w, iv, x);
        if (TWICE) {
#pragma unroll
            for (int j = 0; j < NJ; ++j)
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[j] += v[j].v[k] * x.v[k];
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[NJ] += x.v[k] * x.v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c <= NJ; ++c) {
        const double s = warp_sum((double)acc[c]);
        if (lane == 0) sh[c][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x <= NJ) {
        double s = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) s += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * ldp + threadIdx.x] = s;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, ldp, 0, NJ, h2);
        reduce_partials(partial, gridDim.x, ldp, NJ, 1, nw1);
        __syncthreads();
        if (threadIdx.x == 0) {
            double s2 = *nw1;
            for (int j = 0; j < NJ; ++j) s2 -= h2[j] * h2[j];
            *hn = s2 > 0.0 ? sqrt(s2) : 0.0;
            if (ctl) gmres_arnoldi_update(ctl, jcol, m, h1, h2, hn);
            *counter = 0u;
        }
    }
}

// V_{j+1} = w1 / hn (classical Gram-Schmidt once); zero = 0 when given (another vector than w)
template <typename T>
__global__ void __launch_bounds__(256)
scale_out_kernel(const double* __restrict__ hn, const T* __restrict__ w, T* __restrict__ vout, size_t n,
                 const int* __restrict__ done, T* __restrict__ zero) {
    if (done && *done) return;
    const T inv = T(1.0 / *hn);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        vout[idx] = w[idx] * inv;
        if (zero) zero[idx] = T(0);
    }
}

// V_{j+1} = (w1 - sum_j h2_j V_j) / hn; zero = 0 when given (another vector than w)
template <int NJ, typename T, int VW = 1>
__global__ void __launch_bounds__(256)
axpy_scale_kernel(const T* __restrict__ V, size_t ldv, const double* __restrict__ h2,
                  const double* __restrict__ hn, const T* __restrict__ w, T* __restrict__ vout, size_t n,
                  const int* __restrict__ done, T* __restrict__ zero) {
    if (done && *done) return;
    T hc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) hc[j] = T(__ldg(h2 + j));
    const T inv = T(1.0 / *hn);
    for (size_t iv = blockIdx.x * (size_t)blockDim.x + threadIdx.x; iv < n / VW;
         iv += (size_t)gridDim.x * blockDim.x) {
        Lanes<T, VW> x = load_lanes<T, VW>(w, iv);
        if (zero) {
            Lanes<T, VW> z;
#pragma unroll
            for (int k = 0; k < VW; ++k) z.v[k] = T(0);
            store_lanes<T, VW>(zero, iv, z);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const Lanes<T, VW> v = load_lanes<T, VW>(V + (size_t)j * ldv, iv);
#pragma unroll
            for (int k = 0; k < VW; ++k) x.v[k] -= hc[j] * v.v[k];
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) x.v[k] *= inv;
        store_lanes<T, VW>(vout, iv, x);
    }
}

// Classical Gram-Schmidt twice with the second pass delayed by one Arnoldi step (the DCGS2
// arrangement of Swirydowicz, Langou, Ananthan, Yang and Thomas, "Low synchronization
// Gram-Schmidt and GMRES algorithms", 2021): the step that formed w1 = w - V h1 left its second
// pass v = (w1 - V h2) / hn undone, and the next product was taken of w1 instead of v.  One pass
// over the NJ basis vectors then forms v into vout, the product of v from the product z of w1
// through the Arnoldi relation A V_NJ = V_{NJ+1} H -- A v = (z - V c - c_NJ v) / hn with c = H h2
// (ctl->cdl, formed with the Hessenberg column) -- in place of w1, and the next step's first-pass
// dots V_k . A v for k <= NJ (v the last) into h1n; zero = 0 when given (the next product's output).
template <int NJ, typename T, int VW = 1>
__global__ void __launch_bounds__(kDotThreads)
dcgs_fused_kernel(const T* __restrict__ V, size_t ldv, const double* __restrict__ h2, const double* __restrict__ hn,
                  const GmresCtl* __restrict__ ctl, T* __restrict__ w, const T* __restrict__ z,
                  T* __restrict__ vout, T* __restrict__ zero, size_t n, double* __restrict__ scratch,
                  double* __restrict__ h1n, const int* __restrict__ done) {
    if (done && *done) return;
    constexpr int ldp = NJ + 1;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[NJ + 1][kDotThreads / 32];
    T a[NJ], cc[NJ + 1], acc[NJ + 1];
#pragma unroll
    for (int j = 0; j < NJ; ++j) a[j] = T(__ldg(h2 + j));
#pragma unroll
    for (int j = 0; j <= NJ; ++j) { cc[j] = T(ctl->cdl[j]); acc[j] = T(0); }
    const T inv = T(1.0 / *hn);
    for (size_t iv = blockIdx.x * (size_t)kDotThreads + threadIdx.x; iv < n / VW;
         iv += (size_t)gridDim.x * kDotThreads) {
        Lanes<T, VW> v[NJ];
        Lanes<T, VW> x = load_lanes<T, VW>(w, iv), y = load_lanes<T, VW>(z, iv);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            v[j] = load_lanes<T, VW>(V + (size_t)j * ldv, iv);
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                x.v[k] -= a[j] * v[j].v[k];
                y.v[k] -= cc[j] * v[j].v[k];
            }
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            x.v[k] *= inv;
            y.v[k] = (y.v[k] - cc[NJ] * x.v[k]) * inv;
        }
        store_lanes<T, VW>(vout, iv, x);
        store_lanes<T, VW>(w, iv, y);
        if (zero) {
            Lanes<T, VW> zz;
#pragma unroll
            for (int k = 0; k < VW; ++k) zz.v[k] = T(0);
            store_lanes<T, VW>(zero, iv, zz);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int k = 0; k < VW; ++k) acc[j] += v[j].v[k] * y.v[k];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[NJ] += x.v[k] * y.v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c <= NJ; ++c) {
        const double s = warp_sum((double)acc[c]);
        if (lane == 0) sh[c][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x <= NJ) {
        double s = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) s += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * ldp + threadIdx.x] = s;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, ldp, 0, NJ + 1, h1n);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// ||g||^2 and the residual norms of every candidate initial guess in one pass over g and the
// stored products (no matrix product): out[0] = ||g||^2, out[q] = ||g - sum_j c[q][j] y[j]||^2.
// NQT = the number of stored products (one instance each, the loops bounded by constants).
template <int NQT>
__device__ __forceinline__ void guess_norms_body(size_t n, const double* __restrict__ g, const GuessTerms& t,
                                                 double* __restrict__ scratch, double* __restrict__ out) {
    constexpr int NQ = 7;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[NQ][kDotThreads / 32];
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (size_t idx = blockIdx.x * (size_t)kDotThreads + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * kDotThreads) {
        const double gv = g[idx];
        double yv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) yv[j] = j < NQT ? t.y[j][idx] : 0.0;
        acc[0] += gv * gv;
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            if (q > NQT) break;
            double r = gv;
#pragma unroll
            for (int j = 0; j < 6; ++j)
                if (j < q) r -= t.c[q][j] * yv[j];
            acc[q] += r * r;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double s = warp_sum(acc[q]);
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) s += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, NQ, 0, NQT + 1, out);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// The same norms for the mixed form, whose tolerance is 1e-9 ||g||: the candidates only choose the
// start, and an extrapolated start's norm is then taken exactly.  Every order's coefficients sum to
// one, so g - sum_j c[q][j] y_j = (g - y_0) + sum_{j>=1} c[q][j] (y_0 - y_j): the differences of
// nearly equal vectors are formed first in FP64 (exact when the two are within a factor of two,
// Sterbenz) and rounded once to FP32 (fastcvt.h), which keeps each small difference to FP32
// relative accuracy; the candidates and their squares then run in plain FP32, and the sums across
// threads in FP64.
template <int NQT>
__device__ __forceinline__ void guess_norms_x2_body(size_t n, const double* __restrict__ g, const GuessTerms& t,
                                                    double* __restrict__ scratch, double* __restrict__ out) {
    constexpr int NQ = 7;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[NQ][kDotThreads / 32];
    __shared__ float cf[NQ][6];   // c[q][j] (binomial coefficients: exact in FP32)
    if (threadIdx.x < NQ * 6) cf[threadIdx.x / 6][threadIdx.x % 6] = f64_to_f32(t.c[threadIdx.x / 6][threadIdx.x % 6]);
    __syncthreads();
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    // two entries a grid apart per pass, every load of both issued first; each entry is added
    // to the thread's sums in the order of the one-entry loop
    const size_t stride = (size_t)gridDim.x * kDotThreads;
    for (size_t i0 = blockIdx.x * (size_t)kDotThreads + threadIdx.x; i0 < n; i0 += 2 * stride) {
        double gv[2], yv[2][6];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t idx = i0 + u * stride;
            const bool on = idx < n;
            gv[u] = on ? g[idx] : 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) yv[u][j] = (j < NQT && on) ? t.y[j][idx] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (i0 + u * stride >= n) continue;
            const float gh = f64_to_f32(gv[u]);
            const float e = f64_to_f32(gv[u] - yv[u][0]);   // g - y_0
            float d[6];                                      // y_0 - y_j
            d[0] = 0.f;
#pragma unroll
            for (int j = 1; j < 6; ++j) d[j] = j < NQT ? f64_to_f32(yv[u][0] - yv[u][j]) : 0.f;
            acc[0] = __fmaf_rn(gh, gh, acc[0]);
#pragma unroll
            for (int q = 1; q < NQ; ++q) {
                if (q > NQT) break;
                float r = e;
#pragma unroll
                for (int j = 1; j < 6; ++j)
                    if (j < q) r = __fmaf_rn(cf[q][j], d[j], r);
                acc[q] = __fmaf_rn(r, r, acc[q]);
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double s = warp_sum(f32_to_f64(acc[q]));
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) s += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, NQ, 0, NQT + 1, out);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

template <int NQT>
__global__ void __launch_bounds__(kDotThreads)
guess_norms_kernel(size_t n, const double* __restrict__ g, GuessTerms t, double* __restrict__ scratch,
                   double* __restrict__ out) {
    guess_norms_body<NQT>(n, g, t, scratch, out);
}

template <int NQT>
__global__ void __launch_bounds__(kDotThreads)
guess_norms_x2_kernel(size_t n, const double* __restrict__ g, GuessTerms t, double* __restrict__ scratch,
                      double* __restrict__ out) {
    guess_norms_x2_body<NQT>(n, g, t, scratch, out);
}

// The least-squares start (krylov_guess_ls): over the affine span of the stored solutions,
// written in Newton's backward differences f_p = nabla^p y_0 (y_j = S~ x~_{n-1-j}),
// x0 = x_0 - sum_{p>=1} gamma_p nabla^p x_0 has the residual e + sum_p gamma_p f_p with
// e = g - y_0, and the gamma minimising it solves G gamma = -b, G_pq = f_p . f_q, b_p = f_p . e
// (the polynomial extrapolation through the same solutions is gamma = (-1, ..., -1); the
// differences of successive orders are far from parallel, unlike y_0 - y_j).  One pass over g and
// the NQT stored products gives, with the first differences y_{j-1} - y_j formed in FP64 (exact
// for nearly equal values) and rounded once to FP32, the higher ones and every sum in FP32 per
// thread, FP64 across threads:
//   s[0] = ||g||^2, s[1] = ||e||^2, s[2 + p - 1] = b_p, s[7 + 5 (p-1) + (q-1)] = G_pq (p <= q).
constexpr int kGramSlots = 32;

template <int NQT>
__device__ __forceinline__ void guess_gram_body(size_t n, const double* __restrict__ g, const GuessTerms& t,
                                                double* __restrict__ scratch, double* __restrict__ out) {
    constexpr int D = NQT - 1, NA = 2 + D + D * (D + 1) / 2;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[NA][kDotThreads / 32];
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.f;
    const size_t stride = (size_t)gridDim.x * kDotThreads;
    for (size_t i0 = blockIdx.x * (size_t)kDotThreads + threadIdx.x; i0 < n; i0 += 2 * stride) {
        double gv[2], yv[2][6];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t idx = i0 + u * stride;
            const bool on = idx < n;
            gv[u] = on ? g[idx] : 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) yv[u][j] = (j < NQT && on) ? t.y[j][idx] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (i0 + u * stride >= n) continue;
            const float gh = f64_to_f32(gv[u]);
            const float e = f64_to_f32(gv[u] - yv[u][0]);
            // the difference table: row r holds nabla^(r+1) at y_0, y_1, ...; d[p-1] = nabla^p y_0
            float tab[D > 0 ? D : 1], d[D > 0 ? D : 1];
#pragma unroll
            for (int j = 0; j < D; ++j) tab[j] = f64_to_f32(yv[u][j] - yv[u][j + 1]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                d[r] = tab[0];
#pragma unroll
                for (int j = 0; j + 1 < D - r; ++j) tab[j] = __fsub_rn(tab[j], tab[j + 1]);
            }
            acc[0] = __fmaf_rn(gh, gh, acc[0]);
            acc[1] = __fmaf_rn(e, e, acc[1]);
#pragma unroll
            for (int i = 0; i < D; ++i) acc[2 + i] = __fmaf_rn(d[i], e, acc[2 + i]);
            int a = 2 + D;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = i; j < D; ++j) {
                    acc[a] = __fmaf_rn(d[i], d[j], acc[a]);
                    ++a;
                }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const double v = warp_sum(f32_to_f64(acc[a]));
        if (lane == 0) sh[a][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NA) {
        double v = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) v += sh[threadIdx.x][k];
        partial[(size_t)blockIdx.x * kGramSlots + threadIdx.x] = v;
    }
    if (last_block_arrives(counter)) {
        // the partial columns in their compact order, written to the fixed slots of `out`
        const int lane2 = threadIdx.x & 31, wid2 = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int a = wid2; a < NA; a += nw) {
            double v = strided_sum(partial + a, lane2, 32, gridDim.x, (size_t)kGramSlots, 0.0);
            v = warp_sum(v);
            if (lane2 == 0) {
                int slot = a;   // 0, 1 and the b's keep their index; G_ij goes to 7 + 5 i + j
                if (a >= 2 + D) {
                    int r = a - (2 + D), i = 0;
                    while (r >= D - i) {
                        r -= D - i;
                        ++i;
                    }
                    slot = 7 + 5 * i + (i + r);
                }
                out[slot] = v;
            }
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

template <int NQT>
__global__ void __launch_bounds__(kDotThreads)
guess_gram_kernel(size_t n, const double* __restrict__ g, GuessTerms t, double* __restrict__ scratch,
                  double* __restrict__ out) {
    guess_gram_body<NQT>(n, g, t, scratch, out);
}

__global__ void __launch_bounds__(kDotThreads)
guess_gram_dev_kernel(size_t n, const double* __restrict__ g, const DevHist* __restrict__ dh,
                      double* __restrict__ scratch, double* __restrict__ out) {
    const int avail = dh->avail;
    if (avail <= 0 || avail > 6) return;
    GuessTerms t;
#pragma unroll
    for (int j = 0; j < 6; ++j) t.y[j] = j < avail ? dh->y[j] : nullptr;
    t.nq = avail;
    switch (avail) {
#define CASE(Q) \
    case Q: guess_gram_body<Q>(n, g, t, scratch, out); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
        default: break;
    }
}

// The refinement residual's last pass: w = rhs - (hm + hp) (the two halves of each row of S~ x~,
// minus side first, as mf_sum_kernel) and ||w||^2, 16-byte lanes, grid sum finished by the last block.
__global__ void __launch_bounds__(kDotThreads)
sum_residual_norm_kernel(size_t n, const double* __restrict__ hm, const double* __restrict__ hp,
                         const double* __restrict__ rhs, double* __restrict__ w, double* __restrict__ scratch,
                         double* __restrict__ out) {
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    __shared__ double sh[kDotThreads / 32];
    double acc = 0.0;
    for (size_t iv = blockIdx.x * (size_t)kDotThreads + threadIdx.x; iv < n / 2; iv += (size_t)gridDim.x * kDotThreads) {
        const double2 a = reinterpret_cast<const double2*>(hm)[iv], b = reinterpret_cast<const double2*>(hp)[iv];
        const double2 g = reinterpret_cast<const double2*>(rhs)[iv];
        const double r0 = g.x - (a.x + b.x), r1 = g.y - (a.y + b.y);
        reinterpret_cast<double2*>(w)[iv] = make_double2(r0, r1);
        acc += r0 * r0;
        acc += r1 * r1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {   // an odd last entry
        const double r = rhs[n - 1] - (hm[n - 1] + hp[n - 1]);
        w[n - 1] = r;
        acc += r * r;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double v = warp_sum(acc);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kDotThreads / 32; ++k) t += sh[k];
        partial[blockIdx.x] = t;
    }
    if (last_block_arrives(counter)) {
        reduce_partials(partial, gridDim.x, 1, 0, 1, out);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

struct GuessCoef {
    double c[7][6];
};

// The step graph's form: the history's length and pointers from device memory (DevHist); the
// same sums as the kernels above for that length, nothing when there is no history.
template <bool X2>
__global__ void __launch_bounds__(kDotThreads)
guess_norms_dev_kernel(size_t n, const double* __restrict__ g, const DevHist* __restrict__ dh, GuessCoef cf,
                       double* __restrict__ scratch, double* __restrict__ out) {
    const int avail = dh->avail;
    if (avail <= 0 || avail > 6) return;
    GuessTerms t;
#pragma unroll
    for (int j = 0; j < 6; ++j) t.y[j] = j < avail ? dh->y[j] : nullptr;
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
        for (int j = 0; j < 6; ++j) t.c[q][j] = cf.c[q][j];
    t.nq = avail;
    switch (avail) {
#define CASE(Q)                                                   \
    case Q:                                                       \
        if constexpr (X2) guess_norms_x2_body<Q>(n, g, t, scratch, out); \
        else guess_norms_body<Q>(n, g, t, scratch, out);          \
        break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
        default: break;
    }
}

// ---- device-side GMRES control: one thread each -----------------------------------------
__global__ void gmres_solve_init_kernel(GmresCtl* c, double tol_abs, double inner_rel, int maxit) {
    c->tol_abs = tol_abs;
    c->inner_rel = inner_rel;
    c->maxit = maxit;
    c->total = 0;
    c->status = 0;
}

// Start a restart cycle from the residual whose squared norm is *nrm2.
__global__ void gmres_cycle_init_kernel(GmresCtl* c, const double* nrm2) {
    const double rn = sqrt(*nrm2);
    c->rnorm = rn;
    for (int i = 0; i <= GmresCtl::kM; ++i) c->s[i] = 0.0;
    c->s[0] = rn;
    c->jend = 0;
    c->done = c->total >= c->maxit ? 1 : 0;
    c->tol_cycle = fmax(c->tol_abs, c->inner_rel * rn);
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, Givens rotations, the
// residual estimate |s_{j+1}| and the cycle's stop test (one thread).
__device__ void gmres_arnoldi_update(GmresCtl* c, int j, int m, const double* h1, const double* h2,
                                     const double* hn) {
    if (c->done) return;
    for (int i = 0; i <= j; ++i) c->H[i][j] = c->Hr[i][j] = h1[i] + h2[i];
    c->H[j + 1][j] = c->Hr[j + 1][j] = *hn;
    // c = H h2 over the raw columns 0..j (the delayed second pass's correction of the next product)
    for (int i = 0; i <= j + 1; ++i) {
        double t = 0.0;
        for (int k = i > 0 ? i - 1 : 0; k <= j; ++k) t += c->Hr[i][k] * h2[k];
        c->cdl[i] = t;
    }
    for (int i = 0; i < j; ++i) {
        const double t = c->cs[i] * c->H[i][j] + c->sn[i] * c->H[i + 1][j];
        c->H[i + 1][j] = -c->sn[i] * c->H[i][j] + c->cs[i] * c->H[i + 1][j];
        c->H[i][j] = t;
    }
    const double a = c->H[j][j], b = c->H[j + 1][j];
    const double den = hypot(a, b);
    const double cs = den > 0.0 ? a / den : 1.0, sn = den > 0.0 ? b / den : 0.0;
    c->cs[j] = cs;
    c->sn[j] = sn;
    c->H[j][j] = den;
    c->H[j + 1][j] = 0.0;
    c->s[j + 1] = -sn * c->s[j];
    c->s[j] = cs * c->s[j];
    c->total += 1;
    c->jend = j + 1;
    const double est = fabs(c->s[j + 1]);
    if (!isfinite(est)) { c->status = 1; c->done = 1; return; }
    if (est <= c->tol_cycle || b == 0.0 || c->total >= c->maxit || j == m - 1) c->done = 1;
}

// y = H(0:jend, 0:jend)^{-1} s by back substitution.
__global__ void gmres_solve_y_kernel(GmresCtl* c) {
    for (int i = c->jend - 1; i >= 0; --i) {
        double acc = c->s[i];
        for (int k = i + 1; k < c->jend; ++k) acc -= c->H[i][k] * c->y[k];
        c->y[i] = acc / c->H[i][i];
    }
}

// x += sum_{j < jend} y_j V_j.  FP64 basis: FP64 sums.  FP32 basis (the mixed form's inner
// cycles): the correction is summed in FP32 -- the cycle that produced it is FP32 throughout --
// and added to the FP64 iterate once, one conversion (fastcvt.h) and one FP64 add per entry.
// VW entries per thread (16-byte lanes of FP32 bases); the basis loads are issued four vectors at a
// time and added in their order.
template <typename T, int VW = 1>
__global__ void gmres_update_x_kernel(const T* __restrict__ V, size_t ldv, const GmresCtl* __restrict__ c,
                                      double* __restrict__ x, size_t n) {
    const int nv = c->jend;
    __shared__ T sy[GmresCtl::kM];
    for (int j = threadIdx.x; j < nv; j += blockDim.x) sy[j] = T(c->y[j]);
    __syncthreads();
    for (size_t iv = blockIdx.x * (size_t)blockDim.x + threadIdx.x; iv < n / VW;
         iv += (size_t)gridDim.x * blockDim.x) {
        T acc[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = T(0);
        for (int j0 = 0; j0 < nv; j0 += 4) {
            Lanes<T, VW> v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < nv) v[u] = load_lanes<T, VW>(V + (size_t)(j0 + u) * ldv, iv);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < nv) {
#pragma unroll
                    for (int k = 0; k < VW; ++k) acc[k] += sy[j0 + u] * v[u].v[k];
                }
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) x[iv * VW + k] += to_f64(acc[k]);
    }
}

int stream_grid(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b > 0 ? (int)b : 1;
}

template <int NF>
cudaError_t block_diag_launch(int n_edges, const double* Bd, const double* x, double* y, cudaStream_t s,
                              bool pairs) {
    constexpr int EPB = 256 / NF;
    if (pairs)
        block_diag_x2_kernel<NF><<<(n_edges + EPB - 1) / EPB, EPB * NF, 0, s>>>(
            n_edges, reinterpret_cast<const float2*>(Bd), x, y);
    else
        block_diag_kernel<NF><<<(n_edges + EPB - 1) / EPB, EPB * NF, 0, s>>>(n_edges, Bd, x, y);
    count_launches(1);
    return cudaGetLastError();
}

// 16-byte lanes: FP32 vectors that all start on a 16-byte boundary, n and the basis stride
// multiples of 4
template <typename T>
bool lanes4(size_t n, size_t ldv, std::initializer_list<const void*> ptrs) {
    if (sizeof(T) != 4 || n % 4 != 0 || ldv % 4 != 0) return false;
    for (const void* p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
    return true;
}

// 16-byte lanes of FP64 vectors: every vector on a 16-byte boundary, n and the stride even
template <typename T>
bool lanes2d(size_t n, size_t ldv, std::initializer_list<const void*> ptrs) {
    if (sizeof(T) != 8 || n % 2 != 0 || ldv % 2 != 0) return false;
    for (const void* p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
    return true;
}

template <int NJ, typename T>
cudaError_t cgs2_tail_launch(const T* V, size_t ldv, const double* h1, T* w, size_t n, double* scratch,
                             double* h2, double* nw1, double* hn, T* vout, GmresCtl* ctl, int j, int m,
                             bool twice, cudaStream_t s, const int* done, T* zero) {
    // the NJ x 4 basis lanes stay in registers (80 at NJ = 10: three blocks per SM, hence the grid)
    if constexpr (sizeof(T) == 4 && NJ <= 10) {
        if (twice && lanes4<T>(n, ldv, {V, w, vout, zero ? zero : vout})) {
            axpy_dot_kernel<NJ, T, true, 4><<<152 * 3, kDotThreads, 0, s>>>(V, ldv, h1, w, n, scratch, h2, nw1, hn,
                                                                             ctl, j, m, done);
            axpy_scale_kernel<NJ, T, 4><<<stream_grid(n / 4), 256, 0, s>>>(V, ldv, h2, hn, w, vout, n, done, zero);
            count_launches(2);
            return cudaGetLastError();
        }
    }
    if (twice) {
        axpy_dot_kernel<NJ, T, true><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, h1, w, n, scratch, h2, nw1, hn,
                                                                        ctl, j, m, done);
        count_launches(1);
        axpy_scale_kernel<NJ, T><<<stream_grid(n), 256, 0, s>>>(V, ldv, h2, hn, w, vout, n, done, zero);
    } else {
        axpy_dot_kernel<NJ, T, false><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, h1, w, n, scratch, h2, nw1, hn,
                                                                         ctl, j, m, done);
        count_launches(1);
        scale_out_kernel<T><<<stream_grid(n), 256, 0, s>>>(hn, w, vout, n, done, zero);
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t cgs2_tail_dispatch(const T* V, size_t ldv, int nv, const double* h1, T* w, size_t n,
                               double* scratch, double* h2, double* nw1, double* hn, T* vout,
                               GmresCtl* ctl, int j, int m, bool twice, cudaStream_t s, const int* done,
                               T* zero) {
    switch (nv) {
#define CASE(J) case J: return cgs2_tail_launch<J, T>(V, ldv, h1, w, n, scratch, h2, nw1, hn, vout, ctl, j, m, twice, s, done, zero);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
        CASE(12) CASE(13) CASE(14) CASE(15) CASE(16) CASE(17) CASE(18) CASE(19) CASE(20) CASE(21)
        CASE(22) CASE(23) CASE(24) CASE(25) CASE(26) CASE(27) CASE(28) CASE(29) CASE(30) CASE(31)
        CASE(32)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int NJ>
cudaError_t cgs2_update_launch(const float* V, size_t ldv, const double* h1, float* w, size_t n, double* scratch,
                               double* h2, double* nw1, double* hn, GmresCtl* ctl, int j, int m, cudaStream_t s,
                               const int* done) {
    if constexpr (NJ <= 10) {
        if (lanes4<float>(n, ldv, {V, w})) {
            axpy_dot_kernel<NJ, float, true, 4><<<152 * 3, kDotThreads, 0, s>>>(V, ldv, h1, w, n, scratch, h2, nw1, hn,
                                                                                 ctl, j, m, done);
            count_launches(1);
            return cudaGetLastError();
        }
    }
    axpy_dot_kernel<NJ, float, true><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, h1, w, n, scratch, h2, nw1, hn, ctl, j,
                                                                         m, done);
    count_launches(1);
    return cudaGetLastError();
}

template <int NJ>
cudaError_t dcgs_fused_launch(const float* V, size_t ldv, const double* h2, const double* hn, const GmresCtl* ctl,
                              float* w, const float* z, float* vout, float* zero, size_t n, double* scratch,
                              double* h1n, cudaStream_t s, const int* done) {
    if constexpr (NJ <= 10) {
        if (lanes4<float>(n, ldv, {V, w, z, vout, zero ? zero : vout})) {
            // up to 80 registers a thread through NJ = 8: three blocks per SM; two above
            constexpr int kGrid = 152 * (NJ <= 8 ? 3 : 2);
            dcgs_fused_kernel<NJ, float, 4><<<kGrid, kDotThreads, 0, s>>>(V, ldv, h2, hn, ctl, w, z, vout, zero, n,
                                                                         scratch, h1n, done);
            count_launches(1);
            return cudaGetLastError();
        }
    }
    dcgs_fused_kernel<NJ, float><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, h2, hn, ctl, w, z, vout, zero, n, scratch,
                                                                   h1n, done);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t multidot_impl(const T* V, size_t ldv, int nv, const T* w, size_t n, double* scratch, double* out,
                          cudaStream_t s, const int* done) {
    // one instance per column count: a runtime bound on the column loop would leave predicated-off
    // FMAs in the kernel, and on GB300 those still occupy the slow FP64 pipe
    const bool v4 = lanes4<T>(n, ldv, {V, w});
    const bool v2 = lanes2d<T>(n, ldv, {V, w});
    for (int j0 = 0; j0 < nv; j0 += kDotChunk) {
        const int nj = nv - j0 < kDotChunk ? nv - j0 : kDotChunk;
        switch (nj) {
#define CASE(C)                                                                                                   \
    case C:                                                                                                       \
        if constexpr (sizeof(T) == 4) {                                                                           \
            if (v4) {                                                                                             \
                multidot_kernel<C, T, 4><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, j0, nj, w, n, scratch, nv, out, \
                                                                           done);                                 \
                break;                                                                                            \
            }                                                                                                     \
        } else {                                                                                                  \
            if (v2) {                                                                                             \
                multidot_kernel<C, T, 2><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, j0, nj, w, n, scratch, nv, out, \
                                                                           done);                                 \
                break;                                                                                            \
            }                                                                                                     \
        }                                                                                                         \
        multidot_kernel<C, T><<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, j0, nj, w, n, scratch, nv, out, done);   \
        break;
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace

size_t guess_scratch_doubles() { return 1 + (size_t)kDotBlocks * kGramSlots; }

cudaError_t launch_sum_residual_norm(size_t n, const double* hm, const double* hp, const double* rhs, double* w,
                                     double* scratch, double* out, cudaStream_t s) {
    for (const void* p : {static_cast<const void*>(hm), static_cast<const void*>(hp), static_cast<const void*>(rhs),
                          static_cast<const void*>(w)})
        if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return cudaErrorMisalignedAddress;
    sum_residual_norm_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(n, hm, hp, rhs, w, scratch, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_gram(size_t n, const double* g, const GuessTerms& t, double* scratch, double* out,
                              cudaStream_t s) {
    switch (t.nq) {
#define CASE(Q) \
    case Q: guess_gram_kernel<Q><<<kDotBlocks, kDotThreads, 0, s>>>(n, g, t, scratch, out); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_gram_dev(size_t n, const double* g, const DevHist* dh, double* scratch, double* out,
                                  cudaStream_t s) {
    guess_gram_dev_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(n, g, dh, scratch, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_norms(size_t n, const double* g, const GuessTerms& t, double* scratch, double* out,
                               cudaStream_t s, bool f32x2) {
    switch (t.nq) {
#define CASE(Q)                                                                                   \
    case Q:                                                                                       \
        if (f32x2) guess_norms_x2_kernel<Q><<<kDotBlocks, kDotThreads, 0, s>>>(n, g, t, scratch, out); \
        else guess_norms_kernel<Q><<<kDotBlocks, kDotThreads, 0, s>>>(n, g, t, scratch, out);          \
        break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_norms_dev(size_t n, const double* g, const DevHist* dh, const double (*coef)[6],
                                   double* scratch, double* out, cudaStream_t s, bool f32x2) {
    GuessCoef cf;
    for (int q = 0; q < 7; ++q)
        for (int j = 0; j < 6; ++j) cf.c[q][j] = coef[q][j];
    if (f32x2) guess_norms_dev_kernel<true><<<kDotBlocks, kDotThreads, 0, s>>>(n, g, dh, cf, scratch, out);
    else guess_norms_dev_kernel<false><<<kDotBlocks, kDotThreads, 0, s>>>(n, g, dh, cf, scratch, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cgs2_tail(const double* V, size_t ldv, int nv, const double* h1, double* w, size_t n,
                             double* scratch, double* h2, double* nw1, double* hn, double* vout,
                             GmresCtl* ctl, int j, int m, bool twice, cudaStream_t s, const int* done) {
    return cgs2_tail_dispatch<double>(V, ldv, nv, h1, w, n, scratch, h2, nw1, hn, vout, ctl, j, m, twice, s, done,
                                      nullptr);
}

cudaError_t launch_cgs2_tail(const float* V, size_t ldv, int nv, const double* h1, float* w, size_t n,
                             double* scratch, double* h2, double* nw1, double* hn, float* vout,
                             GmresCtl* ctl, int j, int m, bool twice, cudaStream_t s, const int* done,
                             float* zero) {
    return cgs2_tail_dispatch<float>(V, ldv, nv, h1, w, n, scratch, h2, nw1, hn, vout, ctl, j, m, twice, s, done,
                                     zero);
}

cudaError_t launch_cgs2_update(const float* V, size_t ldv, int nv, const double* h1, float* w, size_t n,
                               double* scratch, double* h2, double* nw1, double* hn, GmresCtl* ctl, int j, int m,
                               cudaStream_t s, const int* done) {
    switch (nv) {
#define CASE(J) case J: return cgs2_update_launch<J>(V, ldv, h1, w, n, scratch, h2, nw1, hn, ctl, j, m, s, done);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
        CASE(12) CASE(13) CASE(14) CASE(15) CASE(16) CASE(17) CASE(18) CASE(19) CASE(20) CASE(21)
        CASE(22) CASE(23) CASE(24) CASE(25) CASE(26) CASE(27) CASE(28) CASE(29) CASE(30) CASE(31)
        CASE(32)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dcgs_fused(const float* V, size_t ldv, int nj, const double* h2, const double* hn,
                              const GmresCtl* ctl, float* w, const float* z, float* vout, float* zero, size_t n,
                              double* scratch, double* h1n, cudaStream_t s, const int* done) {
    switch (nj) {
#define CASE(J) case J: return dcgs_fused_launch<J>(V, ldv, h2, hn, ctl, w, z, vout, zero, n, scratch, h1n, s, done);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
        CASE(12) CASE(13) CASE(14) CASE(15) CASE(16) CASE(17) CASE(18) CASE(19) CASE(20) CASE(21)
        CASE(22) CASE(23) CASE(24) CASE(25) CASE(26) CASE(27) CASE(28) CASE(29) CASE(30) CASE(31)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_block_diag(const Geom& g, const double* Bd, const double* x, double* y,
                              cudaStream_t s, bool pairs) {
    switch (g.P) {
        case 2: return block_diag_launch<6>(g.n_edges, Bd, x, y, s, pairs);
        case 3: return block_diag_launch<9>(g.n_edges, Bd, x, y, s, pairs);
        case 4: return block_diag_launch<12>(g.n_edges, Bd, x, y, s, pairs);
        case 5: return block_diag_launch<15>(g.n_edges, Bd, x, y, s, pairs);
        case 6: return block_diag_launch<18>(g.n_edges, Bd, x, y, s, pairs);
        case 7: return block_diag_launch<21>(g.n_edges, Bd, x, y, s, pairs);
        case 8: return block_diag_launch<24>(g.n_edges, Bd, x, y, s, pairs);
        case 9: return block_diag_launch<27>(g.n_edges, Bd, x, y, s, pairs);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_split_pairs_inplace(double* a, size_t n, cudaStream_t s) {
    split_pairs_inplace_kernel<<<stream_grid(n), 256, 0, s>>>(a, n);
    count_launches(1);
    return cudaGetLastError();
}

size_t dot_scratch_doubles(int nv) { return 1 + (size_t)kDotBlocks * (size_t)nv; }   // ticket + partials

cudaError_t launch_multidot(const double* V, size_t ldv, int nv, const double* w, size_t n,
                            double* scratch, double* out, cudaStream_t s, const int* done) {
    return multidot_impl<double>(V, ldv, nv, w, n, scratch, out, s, done);
}

cudaError_t launch_multidot(const float* V, size_t ldv, int nv, const float* w, size_t n,
                            double* scratch, double* out, cudaStream_t s, const int* done) {
    return multidot_impl<float>(V, ldv, nv, w, n, scratch, out, s, done);
}

cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, double* v, size_t n,
                                  cudaStream_t s) {
    scale_kernel<double><<<stream_grid(n), 256, 0, s>>>(w, nrm2, v, n, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, float* v, size_t n,
                                  cudaStream_t s, float* zero) {
    scale_kernel<float><<<stream_grid(n), 256, 0, s>>>(w, nrm2, v, n, zero);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gmres_solve_init(GmresCtl* c, double tol_abs, double inner_rel, int maxit, cudaStream_t s) {
    gmres_solve_init_kernel<<<1, 1, 0, s>>>(c, tol_abs, inner_rel, maxit);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gmres_cycle_init(GmresCtl* c, const double* nrm2, cudaStream_t s) {
    gmres_cycle_init_kernel<<<1, 1, 0, s>>>(c, nrm2);
    count_launches(1);
    return cudaGetLastError();
}


cudaError_t launch_gmres_update(const double* V, size_t ldv, GmresCtl* c, double* x, size_t n, cudaStream_t s) {
    gmres_solve_y_kernel<<<1, 1, 0, s>>>(c);
    gmres_update_x_kernel<double><<<stream_grid(n), 256, 0, s>>>(V, ldv, c, x, n);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_gmres_update(const float* V, size_t ldv, GmresCtl* c, double* x, size_t n, cudaStream_t s) {
    gmres_solve_y_kernel<<<1, 1, 0, s>>>(c);
    if (lanes4<float>(n, ldv, {V})) gmres_update_x_kernel<float, 4><<<stream_grid(n / 4), 256, 0, s>>>(V, ldv, c, x, n);
    else gmres_update_x_kernel<float><<<stream_grid(n), 256, 0, s>>>(V, ldv, c, x, n);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* a, float* b, size_t n, cudaStream_t s) {
    to_f32_kernel<<<stream_grid(n), 256, 0, s>>>(a, b, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hdgdg
