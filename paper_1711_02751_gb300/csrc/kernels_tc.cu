// Shared-operator local contractions on the 5th-generation tensor cores (tcgen05).
//
// With a flat bottom and one time step, every element has the same local operator A (eq.
// linearizedHDGsystem: A = I - dt a_ii M^{-1} dL/dQ depends only on phi_B, tau and the
// reference element), so the condensation Z = A^{-1} R1 and the recovery A^{-1}(tau qhat) of all
// elements are ONE dense product
//
//     D [elements x NV] = X [elements x NV] * (A^{-1})^T,      NV = 3 (k+1)^2,
//
// with X the rows R1_e (condensation) or the boundary values tau qhat gathered per element
// (recovery, zero at interior nodes).  One CTA of 128 threads takes 128 elements:
//   * warp 0 allocates tensor memory for the 128 x NPAD FP32 accumulator;
//   * thread 0 starts a bulk copy (TMA) of the operator tile (BF16, prepared once at setup in
//     the tensor core's shared-memory layout) into shared memory;
//   * all threads write X's 128 rows as BF16 into shared memory in the same layout;
//   * thread 0 issues KP/16 tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulate, M = 128,
//     N = NPAD) and commits them to an mbarrier;
//   * every warp reads its 32 accumulator rows back with tcgen05.ld into a shared-memory tile,
//     and the CTA writes the FP64 result field plane by field plane with consecutive threads
//     on consecutive addresses (in recovery also reading Z and R1 that way: Q = Z + beta D,
//     L_i = (Q - R1)/a_ii).
// Every wait is bounded: when one runs out the kernel sets *error, skips the dependent work,
// frees its tensor memory and returns.
//
// Shared-memory operand layout (no swizzle, K-major): the matrix is cut into core matrices of
// 8 rows x 16 bytes (8 BF16 values along K) stored as 128 contiguous bytes; core matrices
// adjacent along K are 128 bytes apart (leading byte offset) and 8-row groups are KP*16 bytes
// apart (stride byte offset).  Rows beyond the valid elements and columns beyond NV are zero.
#include <cuda_bf16.h>
#include <cstdint>

#include "async_copy.h"
#include "internal.h"

namespace hdgdg {
namespace {

constexpr int kTileM = 128;          // elements per CTA = accumulator lanes
constexpr int kThreads = 128;

__host__ __device__ constexpr int pad16(int n) { return (n + 15) / 16 * 16; }
__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

template <int P>
struct TcShape {
    static constexpr int Np = P * P, NV = 3 * Np;
    static constexpr int KP = pad16(NV);       // K padded to the BF16 MMA step (16)
    static constexpr int NPAD = pad16(NV);     // N: a multiple of 16 for M = 128
    static constexpr int COLS = tmem_cols(NPAD);
    static constexpr int A_BYTES = kTileM * KP * 2;
    static constexpr int B_BYTES = NPAD * KP * 2;
    static constexpr int SBO = KP * 16;        // bytes between 8-row groups
    static constexpr int DS = NV | 1;          // row stride (floats) of the staged result: odd, no bank conflicts
    static constexpr int D_BYTES = kTileM * DS * 4;
};

// byte offset of (row, k) in the canonical K-major layout above
__host__ __device__ inline int tile_offset(int row, int k, int sbo) {
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// warp-wide: allocate `cols` tensor-memory columns, base address written to *holder
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset >> 4 (16-29),
// stride byte offset >> 4 (32-45), descriptor version 1 (46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    const uint64_t a = (smem_addr(p) >> 4) & 0x3FFF;
    return a | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's accumulator row (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void store_bf16(uint8_t* tile, int row, int k, int sbo, double v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + tile_offset(row, k, sbo)) = __double2bfloat16(v);
}

// Setup: the shared operator's tile from element 0's FP64 A^{-1} (column major).
template <int P>
__global__ void tc_image_kernel(const double* __restrict__ Ainv, uint8_t* __restrict__ image) {
    using S = TcShape<P>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S::NPAD * S::KP) return;
    const int r = t / S::KP, k = t % S::KP;   // B row = output index r, column = input index k
    const double v = (r < S::NV && k < S::NV) ? Ainv[(size_t)k * S::NV + r] : 0.0;
    *reinterpret_cast<__nv_bfloat16*>(image + tile_offset(r, k, S::SBO)) = __double2bfloat16(v);
}

template <int P, int MODE>
__global__ void __launch_bounds__(kThreads) local_tc_kernel(
    Geom g, const uint8_t* __restrict__ image, const double* __restrict__ R1, const double* __restrict__ Z,
    const double* __restrict__ tau_edge, const double* __restrict__ qhat, double beta, double inv_aii,
    double* __restrict__ out0, double* __restrict__ out1, int* __restrict__ error) {
    using S = TcShape<P>;
    constexpr int Np = S::Np, NV = S::NV, NF = 3 * P;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sA = smem;                  // 128 x KP BF16 rows of X
    uint8_t* sB = smem + S::A_BYTES;     // NPAD x KP BF16 operator tile
    float* sD = reinterpret_cast<float*>(smem + S::A_BYTES + S::B_BYTES);   // 128 x DS FP32 result
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_holder;
    __shared__ int s_issued;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int e0 = blockIdx.x * kTileM;
    const int cnt = min(kTileM, g.n_el - e0);
    const size_t fs = (size_t)g.n_el * Np;

    if (warp == 0) tmem_alloc(&tmem_holder, S::COLS);
    if (tid == 0) {
        mbar_init(&bar_tma, 1);
        mbar_init(&bar_mma, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < S::A_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    if (tid == 0) {
        mbar_expect_tx(&bar_tma, S::B_BYTES);
        bulk_copy_g2s(sB, image, S::B_BYTES, &bar_tma);
    }

    // X rows (BF16).  Condensation: R1, read coalesced field by field.
    if (MODE == 0) {
        for (int c = 0; c < 3; ++c) {
            const double* src = R1 + c * fs + (size_t)e0 * Np;
            for (int i = tid; i < cnt * Np; i += kThreads) store_bf16(sA, i / Np, c * Np + i % Np, S::SBO, src[i]);
        }
    } else if (tid < cnt) {
        // Recovery: tau qhat summed onto the boundary nodes of element e (corners get two faces).
        const int e = e0 + tid;
        double u[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) u[i] = 0.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int ed = edge_of_face(e, f, g);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const int n = face_node(f, b, P);
                const double tau = tau_edge[(size_t)ed * P + b];
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c * Np + n] += tau * qhat[(size_t)ed * NF + c * P + b];
            }
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) store_bf16(sA, tid, i, S::SBO, u[i]);
    }
    fence_proxy_async();
    __syncthreads();

    if (tid == 0) {
        tc_fence_after();
        int issued = 0;
        if (mbar_wait_bounded(&bar_tma, 0)) {
            constexpr uint32_t idesc = idesc_bf16(kTileM, S::NPAD);
#pragma unroll
            for (int kc = 0; kc < S::KP / 16; ++kc) {
                const uint64_t da = smem_desc(sA + kc * 256, 128, S::SBO);
                const uint64_t db = smem_desc(sB + kc * 256, 128, S::SBO);
                mma_bf16(tmem, da, db, idesc, kc > 0 ? 1u : 0u);
            }
            mma_commit(&bar_mma);
            issued = 1;
        } else {
            atomicExch(error, 1);
        }
        s_issued = issued;
    }
    __syncthreads();
    bool ok = s_issued != 0;
    if (ok) ok = mbar_wait_bounded(&bar_mma, 0);
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0 && s_issued) atomicExch(error, 2);
    tc_fence_after();

    if (ok) {
#pragma unroll
        for (int c0 = 0; c0 < S::NPAD; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < NV) sD[tid * S::DS + c0 + j] = v[j];
        }
    }
    __syncthreads();
    if (ok) {
        for (int c = 0; c < 3; ++c) {
            const size_t base = c * fs + (size_t)e0 * Np;
            for (int i = tid; i < cnt * Np; i += kThreads) {
                const int m = i / Np, n = i % Np;
                const double d = (double)sD[m * S::DS + c * Np + n];
                if (MODE == 0) {
                    out0[base + i] = d;
                } else {
                    const double q = Z[base + i] + beta * dt_factor(g, e0 + m) * d;
                    out0[base + i] = q;
                    out1[base + i] = (q - R1[base + i]) * inv_aii;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, S::COLS);
    }
}

// ---- FP64-class products from BF16 slices (the Ozaki splitting) -------------------------------
// Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012) split each operand into slices so that
// the slices' products are error free in the unit's accumulator.  Here every X row (element) and
// every operator column is scaled by a power of two to |v| < 1 and cut into SL slices of seven bits
// (each an integer |t| <= 128 -- exact in BF16), v = 2^e sum_i t_i 2^{-7(i+1)}.  A product of two
// slices is an integer below 2^14 and a row of K <= 80 of them, over the <= SL pairs (i, j) with
// i + j = s, stays below 2^23: the tensor core's FP32 accumulator D_s holds it exactly.  The pairs
// with i + j >= SL (below 2^{-7 SL} of the result's scale) are left out, so the result carries about
// 7 SL bits; the epilogue adds the D_s with their weights 2^{7(SL-1-s)} in 64-bit integers (exact
// below 2^53) and scales by 2^{e_row + e_col - 7(SL+1)} in FP64.
constexpr int kSlices = 5;   // about 35 bits: 3e-11 relative to the row and column scales

template <int P>
struct TcSplit {
    using S = TcShape<P>;
    static constexpr int IMG = kSlices * S::B_BYTES;            // the operator's slices
    static constexpr int SCALE_OFF = IMG;                       // then NPAD int column exponents
    static constexpr int IMAGE_BYTES = IMG + S::NPAD * 4;
    static constexpr int COLS_USED = kSlices * S::NPAD;
    static constexpr int COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                               : COLS_USED <= 256 ? 256 : 512;
    static constexpr int AS_BYTES = kSlices * S::A_BYTES;       // the X slices (reused for the FP64 result)
    static constexpr int DD = S::NV | 1;                        // row stride (doubles) of the staged result
};

// exponent e with |v| < 2^e for the largest |v| of a set (0 for an all-zero set)
__device__ __forceinline__ int exp_above(double v) {
    int e = 0;
    (void)frexp(v, &e);
    return v == 0.0 ? -1074 : e;
}

// slice v (|v| < 2^e) into kSlices seven-bit integers; t[i] the i-th
__device__ __forceinline__ void split7(double v, int e, float* t) {
    double u = ldexp(v, -e);
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        const double w = u * 128.0;
        const double r = rint(w);
        t[i] = (float)r;
        u = w - r;
    }
}

__device__ __forceinline__ void store_slice(uint8_t* tile, int slice_bytes, int row, int k, int sbo, const float* t) {
#pragma unroll
    for (int i = 0; i < kSlices; ++i)
        *reinterpret_cast<__nv_bfloat16*>(tile + i * slice_bytes + tile_offset(row, k, sbo)) = __float2bfloat16_rn(t[i]);
}

// Setup: the shared operator's slices and column exponents (one thread per output column r).
template <int P>
__global__ void tc_split_image_kernel(const double* __restrict__ Ainv, uint8_t* __restrict__ image) {
    using S = TcShape<P>;
    using Q = TcSplit<P>;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S::NPAD) return;
    double m = 0.0;
    for (int k = 0; k < S::NV && r < S::NV; ++k) m = fmax(m, fabs(Ainv[(size_t)k * S::NV + r]));
    const int e = exp_above(m);
    reinterpret_cast<int*>(image + Q::SCALE_OFF)[r] = e;
    for (int k = 0; k < S::KP; ++k) {
        float t[kSlices];
        const double v = (r < S::NV && k < S::NV) ? Ainv[(size_t)k * S::NV + r] : 0.0;
        split7(v, e < -1000 ? 0 : e, t);
        store_slice(image, S::B_BYTES, r, k, S::SBO, t);
    }
}

template <int P, int MODE>
__global__ void __launch_bounds__(kThreads) local_tc_split_kernel(
    Geom g, const uint8_t* __restrict__ image, const double* __restrict__ R1, const double* __restrict__ Z,
    const double* __restrict__ tau_edge, const double* __restrict__ qhat, double beta, double inv_aii,
    double* __restrict__ out0, double* __restrict__ out1, int* __restrict__ error) {
    using S = TcShape<P>;
    using Q = TcSplit<P>;
    constexpr int Np = S::Np, NV = S::NV, NF = 3 * P;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sA = smem;                        // kSlices x (128 x KP) BF16 slices of X
    uint8_t* sB = smem + Q::AS_BYTES;          // the operator image: kSlices x (NPAD x KP) + exponents
    const int* sEc = reinterpret_cast<const int*>(sB + Q::SCALE_OFF);
    double* sD = reinterpret_cast<double*>(smem);   // 128 x DD FP64 result (over the X slices, after the MMAs)
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_holder;
    __shared__ int s_issued;
    __shared__ int sEr[kTileM];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int e0 = blockIdx.x * kTileM;
    const int cnt = min(kTileM, g.n_el - e0);
    const size_t fs = (size_t)g.n_el * Np;

    if (warp == 0) tmem_alloc(&tmem_holder, Q::COLS);
    if (tid == 0) {
        mbar_init(&bar_tma, 1);
        mbar_init(&bar_mma, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < Q::AS_BYTES / 16; i += kThreads) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
    sEr[tid] = -1074;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    if (tid == 0) {
        mbar_expect_tx(&bar_tma, Q::IMAGE_BYTES);
        bulk_copy_g2s(sB, image, Q::IMAGE_BYTES, &bar_tma);
    }

    if (MODE == 0) {   // condensation: R1 rows, row exponents first, then the slices
        for (int c = 0; c < 3; ++c) {
            const double* src = R1 + c * fs + (size_t)e0 * Np;
            for (int i = tid; i < cnt * Np; i += kThreads) atomicMax(&sEr[i / Np], exp_above(fabs(src[i])));
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) {
            const double* src = R1 + c * fs + (size_t)e0 * Np;
            for (int i = tid; i < cnt * Np; i += kThreads) {
                const int row = i / Np, e = sEr[row];
                float t[kSlices];
                split7(src[i], e < -1000 ? 0 : e, t);
                store_slice(sA, S::A_BYTES, row, c * Np + i % Np, S::SBO, t);
            }
        }
    } else if (tid < cnt) {   // recovery: tau qhat on the boundary nodes of element e (one row per thread)
        const int e = e0 + tid;
        double u[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) u[i] = 0.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int ed = edge_of_face(e, f, g);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const int n = face_node(f, b, P);
                const double tau = tau_edge[(size_t)ed * P + b];
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c * Np + n] += tau * qhat[(size_t)ed * NF + c * P + b];
            }
        }
        double m = 0.0;
#pragma unroll
        for (int i = 0; i < NV; ++i) m = fmax(m, fabs(u[i]));
        const int e_r = exp_above(m);
        sEr[tid] = e_r;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float t[kSlices];
            split7(u[i], e_r < -1000 ? 0 : e_r, t);
            store_slice(sA, S::A_BYTES, tid, i, S::SBO, t);
        }
    }
    fence_proxy_async();
    __syncthreads();

    if (tid == 0) {   // D_s = sum over i + j = s of X_i B_j^T, exact in FP32
        tc_fence_after();
        int issued = 0;
        if (mbar_wait_bounded(&bar_tma, 0)) {
            constexpr uint32_t idesc = idesc_bf16(kTileM, S::NPAD);
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl) {
                bool first = true;
                for (int i = 0; i <= sl; ++i) {
                    const int j = sl - i;
#pragma unroll
                    for (int kc = 0; kc < S::KP / 16; ++kc) {
                        const uint64_t da = smem_desc(sA + i * S::A_BYTES + kc * 256, 128, S::SBO);
                        const uint64_t db = smem_desc(sB + j * S::B_BYTES + kc * 256, 128, S::SBO);
                        mma_bf16(tmem + (uint32_t)(sl * S::NPAD), da, db, idesc, first ? 0u : 1u);
                        first = false;
                    }
                }
            }
            mma_commit(&bar_mma);
            issued = 1;
        } else {
            atomicExch(error, 1);
        }
        s_issued = issued;
    }
    __syncthreads();
    bool ok = s_issued != 0;
    if (ok) ok = mbar_wait_bounded(&bar_mma, 0);
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0 && s_issued) atomicExch(error, 2);
    tc_fence_after();

    // each thread combines its row: V = sum_s D_s 2^{7(SL-1-s)} (integers), then the scales
    if (ok) {
        const int er = sEr[tid];
#pragma unroll
        for (int c0 = 0; c0 < S::NPAD; c0 += 16) {
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * S::NPAD + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = acc[j] * 128 + (long long)v[j];
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = c0 + j;
                if (col < NV) {
                    const int ec = sEc[col];
                    const double d = (er < -1000 || ec < -1000) ? 0.0 : ldexp((double)acc[j], er + ec - 7 * (kSlices + 1));
                    sD[tid * Q::DD + col] = d;
                }
            }
        }
    }
    __syncthreads();
    if (ok) {
        for (int c = 0; c < 3; ++c) {
            const size_t base = c * fs + (size_t)e0 * Np;
            for (int i = tid; i < cnt * Np; i += kThreads) {
                const int m = i / Np, n = i % Np;
                const double d = sD[m * Q::DD + c * Np + n];
                if (MODE == 0) {
                    out0[base + i] = d;
                } else {
                    const double q = Z[base + i] + beta * dt_factor(g, e0 + m) * d;
                    out0[base + i] = q;
                    out1[base + i] = (q - R1[base + i]) * inv_aii;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Q::COLS);
    }
}

template <int P>
size_t split_smem_bytes() {
    using S = TcShape<P>;
    using Q = TcSplit<P>;
    const int max_ctas = 512 / Q::COLS;
    const int d_bytes = kTileM * Q::DD * 8;
    const int need = (Q::AS_BYTES > d_bytes ? Q::AS_BYTES : d_bytes) + Q::IMAGE_BYTES;
    const int floor_bytes = 232448 / max_ctas - 2048;
    return (size_t)(need > floor_bytes ? need : floor_bytes);
}

template <int P>
cudaError_t local_tc_split_launch(const Geom& g, int mode, const void* image, const double* R1, const double* Z,
                                  const double* tau_edge, const double* qhat, double beta, double inv_aii,
                                  double* out0, double* out1, int* error, cudaStream_t s) {
    const size_t smem = split_smem_bytes<P>();
    const int blocks = (g.n_el + kTileM - 1) / kTileM;
    if (mode == 0) {
        cudaError_t e = cudaFuncSetAttribute(local_tc_split_kernel<P, 0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        local_tc_split_kernel<P, 0><<<blocks, kThreads, smem, s>>>(g, static_cast<const uint8_t*>(image), R1, Z,
                                                                   tau_edge, qhat, beta, inv_aii, out0, out1, error);
    } else {
        cudaError_t e = cudaFuncSetAttribute(local_tc_split_kernel<P, 1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        local_tc_split_kernel<P, 1><<<blocks, kThreads, smem, s>>>(g, static_cast<const uint8_t*>(image), R1, Z,
                                                                   tau_edge, qhat, beta, inv_aii, out0, out1, error);
    }
    count_launches(1);
    return cudaGetLastError();
}

template <int P>
size_t smem_bytes() {
    using S = TcShape<P>;
    // at most 512 / COLS CTAs per SM may hold tensor memory at once: ask for enough shared memory
    // that no more than that many are resident
    const int max_ctas = 512 / S::COLS;
    const int need = S::A_BYTES + S::B_BYTES + S::D_BYTES;
    const int floor_bytes = 232448 / max_ctas - 2048;   // 227 KB usable per SM, 1 KB reserved per CTA
    return (size_t)(need > floor_bytes ? need : floor_bytes);
}

template <int P>
cudaError_t local_tc_launch(const Geom& g, int mode, const void* image, const double* R1, const double* Z,
                            const double* tau_edge, const double* qhat, double beta, double inv_aii, double* out0,
                            double* out1, int* error, cudaStream_t s) {
    const size_t smem = smem_bytes<P>();
    const int blocks = (g.n_el + kTileM - 1) / kTileM;
    if (mode == 0) {
        cudaError_t e = cudaFuncSetAttribute(local_tc_kernel<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        local_tc_kernel<P, 0><<<blocks, kThreads, smem, s>>>(g, static_cast<const uint8_t*>(image), R1, Z,
                                                             tau_edge, qhat, beta, inv_aii, out0, out1, error);
    } else {
        cudaError_t e = cudaFuncSetAttribute(local_tc_kernel<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        local_tc_kernel<P, 1><<<blocks, kThreads, smem, s>>>(g, static_cast<const uint8_t*>(image), R1, Z,
                                                             tau_edge, qhat, beta, inv_aii, out0, out1, error);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

size_t tc_image_bytes(int P) {
    const int NV = 3 * P * P;
    return (size_t)pad16(NV) * pad16(NV) * 2;
}

size_t tc_split_image_bytes(int P) {
    switch (P) {
        case 2: return TcSplit<2>::IMAGE_BYTES;
        case 3: return TcSplit<3>::IMAGE_BYTES;
        case 4: return TcSplit<4>::IMAGE_BYTES;
        case 5: return TcSplit<5>::IMAGE_BYTES;
        default: return 0;
    }
}

cudaError_t launch_tc_split_image(const Geom& g, const double* Ainv, void* image, cudaStream_t s) {
#define CALL(P)                                                                                      \
    do {                                                                                             \
        tc_split_image_kernel<P><<<1, 128, 0, s>>>(Ainv, static_cast<uint8_t*>(image));             \
        count_launches(1);                                                                           \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (g.P) {
        case 2: CALL(2);
        case 3: CALL(3);
        case 4: CALL(4);
        case 5: CALL(5);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_local_tc_split(const Geom& g, int mode, const void* image, const double* R1, const double* Z,
                                  const double* tau_edge, const double* qhat, double beta, double inv_aii,
                                  double* out0, double* out1, int* error, cudaStream_t s) {
#define CALL(P) \
    return local_tc_split_launch<P>(g, mode, image, R1, Z, tau_edge, qhat, beta, inv_aii, out0, out1, error, s)
    switch (g.P) {
        case 2: CALL(2);
        case 3: CALL(3);
        case 4: CALL(4);
        case 5: CALL(5);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_tc_image(const Geom& g, const double* Ainv, void* image, cudaStream_t s) {
#define CALL(P)                                                                                         \
    do {                                                                                                \
        const int n = TcShape<P>::NPAD * TcShape<P>::KP;                                              \
        tc_image_kernel<P><<<(n + 255) / 256, 256, 0, s>>>(Ainv, static_cast<uint8_t*>(image));      \
        count_launches(1);                                                                              \
        return cudaGetLastError();                                                                      \
    } while (0)
    switch (g.P) {
        case 2: CALL(2);
        case 3: CALL(3);
        case 4: CALL(4);
        case 5: CALL(5);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_local_tc(const Geom& g, int mode, const void* image, const double* R1, const double* Z,
                            const double* tau_edge, const double* qhat, double beta, double inv_aii, double* out0,
                            double* out1, int* error, cudaStream_t s) {
#define CALL(P) return local_tc_launch<P>(g, mode, image, R1, Z, tau_edge, qhat, beta, inv_aii, out0, out1, error, s)
    switch (g.P) {
        case 2: CALL(2);
        case 3: CALL(3);
        case 4: CALL(4);
        case 5: CALL(5);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace hdgdg
