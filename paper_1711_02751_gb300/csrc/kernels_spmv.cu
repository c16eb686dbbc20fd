// Trace-matrix products of the Krylov solve (Sec. 6, eq. linearizedHDGsystem_schur): y = x + sum
// over the six off-diagonal blocks of the block-Jacobi-preconditioned trace matrix S~ (its
// diagonal blocks are the identity and are not stored) applied to the neighbouring traces.
//   spmv_pre_kernel<NF, T>  one thread per row component; the row's six neighbour trace vectors
//                           are gathered into shared memory first (six independent loads per
//                           thread), then the products read them from there;
//   residual_norm_x2_kernel<NF>  w = g - (x + S~ x) and ||w||^2 in FP64-class arithmetic on the
//                           FP32 pipes (compensated.h): the refinement's true residual;
//   spmv_stream_kernel<NF>  FP32, the matrix also streamed through shared memory by bulk copies.
#include <algorithm>

#include "async_copy.h"
#include "compensated.h"
#include "internal.h"
#include "reduce.h"

namespace hdgdg {
namespace {

// y[r][ii] = x[r][ii] + sum_{slot, jj} S~[r][slot][jj][ii] x[col(r,slot)][jj]
template <int NF, typename T>
__global__ void __launch_bounds__(256)
spmv_pre_kernel(int n_edges, const T* __restrict__ Stil, const int* __restrict__ Scol,
                const T* __restrict__ x, T* __restrict__ y, const int* __restrict__ done) {
    if (done && *done) return;
    constexpr int EPB = 256 / NF;
    __shared__ T sx[EPB][6][NF];   // the six gathered neighbour trace vectors of each edge row
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = blockIdx.x * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) {   // each thread loads one value per slot: six independent loads
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) sx[le][sl][ii] = x[(size_t)__ldg(Scol + (size_t)r * 6 + sl) * NF + ii];
    }
    __syncthreads();
    if (!live) return;
    const T* S = Stil + (size_t)r * 6 * NF * NF;
    T acc = x[(size_t)r * NF + ii];
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) {
        const T* Sb = S + sl * NF * NF;
#pragma unroll
        for (int jj = 0; jj < NF; ++jj) acc += Sb[jj * NF + ii] * sx[le][sl][jj];
    }
    y[(size_t)r * NF + ii] = acc;
}

// w = g - (x + S~ x) with S~ as an FP32 pair (compensated Dot2 sums, compensated.h), and
// ||w||^2: the refinement's true residual and its norm in one pass.  One block per group of EPB
// edge rows (as spmv_pre_kernel); each block leaves its partial sum of squares in scratch and the
// last block to arrive sums them in block order (fixed order, reproducible).
template <int NF>
__global__ void __launch_bounds__(256)
residual_norm_x2_kernel(int n_edges, const float* __restrict__ Shi, const float* __restrict__ Slo,
                        const int* __restrict__ Scol, const double* __restrict__ x, const double* __restrict__ g,
                        double* __restrict__ w, double* __restrict__ scratch, double* __restrict__ nrm2) {
    constexpr int EPB = 256 / NF;
    __shared__ float sxh[EPB][6][NF], sxl[EPB][6][NF];
    __shared__ double sh[8];
    const int le = threadIdx.x / NF, ii = threadIdx.x % NF;
    const int r = blockIdx.x * EPB + le;
    const bool live = le < EPB && r < n_edges;
    if (live) {
#pragma unroll
        for (int sl = 0; sl < 6; ++sl)
            split(x[(size_t)__ldg(Scol + (size_t)r * 6 + sl) * NF + ii], sxh[le][sl][ii], sxl[le][sl][ii]);
    }
    __syncthreads();
    double v2 = 0.0;
    if (live) {
        const size_t base = (size_t)r * 6 * NF * NF;
        Dot2 acc;
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
#pragma unroll
            for (int jj = 0; jj < NF; ++jj) {
                const size_t o = base + (size_t)sl * NF * NF + jj * NF + ii;
                acc.add(Shi[o], Slo[o], sxh[le][sl][jj], sxl[le][sl][jj]);
            }
        }
        const size_t o = (size_t)r * NF + ii;
        const double v = g[o] - (x[o] + acc.value());
        w[o] = v;
        v2 = v * v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double s = warp_sum(v2);
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + 1;
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) b += sh[k];
        partial[blockIdx.x] = b;
    }
    if (last_block_arrives(counter)) {   // the whole block sums the partials, fixed order
        double t = strided_sum(partial, threadIdx.x, blockDim.x, gridDim.x, 1, 0.0);
        t = warp_sum(t);
        __syncthreads();
        if (lane == 0) sh[wid] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) b += sh[k];
            *nrm2 = b;
            *counter = 0u;
        }
    }
}

// The same product with the matrix streamed through shared memory: a persistent CTA takes
// tiles of ET consecutive edge rows; their 6 NF x NF blocks are contiguous in S~, so one bulk
// (TMA) copy per tile brings them in, two stages deep on mbarriers, while the threads (one per
// row component, as above) multiply the previous tile.  Same summation order as
// spmv_pre_kernel, so the results are identical bit for bit.  n_edges * NF must be even (every
// tile a multiple of 16 bytes); a wait that runs out sets *error and ends the CTA.
template <int NF>
struct SpmvTile {
    static constexpr int BLK = 6 * NF * NF;   // floats of one edge row
    static constexpr int ET0 = 55296 / (BLK * 4);
    static constexpr int ET = ET0 > 32 ? 32 : (ET0 < 2 ? 2 : (ET0 & ~1));   // even
    static constexpr int TILE = ET * BLK;
    static constexpr int THREADS = ET * NF;
};

template <int NF>
__global__ void __launch_bounds__(SpmvTile<NF>::THREADS)
spmv_stream_kernel(int n_edges, const float* __restrict__ Stil, const int* __restrict__ Scol,
                   const float* __restrict__ x, float* __restrict__ y, const int* __restrict__ done,
                   int* __restrict__ error) {
    if (done && *done) return;
    using Tl = SpmvTile<NF>;
    extern __shared__ __align__(128) float stile[];     // [2][TILE]
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ float sx[Tl::ET][6][NF];
    const int tid = threadIdx.x;
    const int n_tiles = (n_edges + Tl::ET - 1) / Tl::ET;
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], blockDim.x);
        mbar_init(&empty[1], blockDim.x);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int i) {   // thread 0: the i-th tile of this CTA into stage i % 2
        const int t = blockIdx.x + i * gridDim.x;
        if (t >= n_tiles) return;
        const int e0 = t * Tl::ET;
        const int ne = min(Tl::ET, n_edges - e0);
        const uint32_t bytes = (uint32_t)ne * Tl::BLK * 4u;
        mbar_expect_tx(&full[i & 1], bytes);
        bulk_copy_g2s(stile + (i & 1) * Tl::TILE, Stil + (size_t)e0 * Tl::BLK, bytes, &full[i & 1]);
    };
    if (tid == 0) {
        issue(0);
        issue(1);
    }
    const int le = tid / NF, ii = tid % NF;
    for (int i = 0;; ++i) {
        const int t = blockIdx.x + i * gridDim.x;
        if (t >= n_tiles) break;
        const int st = i & 1;
        const uint32_t parity = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait_bounded(&full[st], parity)) {
            atomicExch(error, 1);
            return;
        }
        const int r = t * Tl::ET + le;
        if (r < n_edges) {   // gather the neighbour trace vectors: six independent loads
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) sx[le][sl][ii] = x[(size_t)__ldg(Scol + (size_t)r * 6 + sl) * NF + ii];
        }
        __syncthreads();
        if (r < n_edges) {
            const float* S = stile + st * Tl::TILE + le * Tl::BLK;
            float acc = x[(size_t)r * NF + ii];
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) {
                const float* Sb = S + sl * NF * NF;
#pragma unroll
                for (int jj = 0; jj < NF; ++jj) acc += Sb[jj * NF + ii] * sx[le][sl][jj];
            }
            y[(size_t)r * NF + ii] = acc;
        }
        __syncthreads();   // sx is rewritten for the next tile
        mbar_arrive(&empty[st]);
        if (tid == 0 && blockIdx.x + (i + 2) * gridDim.x < n_tiles) {
            // the stage is reused for tile i + 2 once every thread has read tile i
            if (!mbar_wait_bounded(&empty[st], parity)) {
                atomicExch(error, 2);
                return;
            }
            issue(i + 2);
        }
    }
}

template <int NF, typename T>
cudaError_t spmv_launch(int n_edges, const T* Stil, const int* Scol, const T* x, T* y, cudaStream_t s,
                        const int* done) {
    constexpr int EPB = 256 / NF;
    spmv_pre_kernel<NF, T><<<(n_edges + EPB - 1) / EPB, EPB * NF, 0, s>>>(n_edges, Stil, Scol, x, y, done);
    count_launches(1);
    return cudaGetLastError();
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        n = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 1;
    }
    return n;
}

template <int NF>
cudaError_t spmv_stream_launch(int n_edges, const float* Stil, const int* Scol, const float* x, float* y,
                               cudaStream_t s, const int* done, int* error) {
    using Tl = SpmvTile<NF>;
    const size_t smem = 2 * (size_t)Tl::TILE * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(spmv_stream_kernel<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int n_tiles = (n_edges + Tl::ET - 1) / Tl::ET;
    const int grid = std::min(n_tiles, 2 * sm_count());   // persistent: two CTAs per SM
    spmv_stream_kernel<NF><<<grid, Tl::THREADS, smem, s>>>(n_edges, Stil, Scol, x, y, done, error);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t spmv_dispatch(const Geom& g, const T* Stil, const int* Scol, const T* x, T* y, cudaStream_t s,
                          const int* done) {
    switch (g.P) {
        case 2: return spmv_launch<6, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 3: return spmv_launch<9, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 4: return spmv_launch<12, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 5: return spmv_launch<15, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 6: return spmv_launch<18, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 7: return spmv_launch<21, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 8: return spmv_launch<24, T>(g.n_edges, Stil, Scol, x, y, s, done);
        case 9: return spmv_launch<27, T>(g.n_edges, Stil, Scol, x, y, s, done);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_spmv_pre(const Geom& g, const double* Stil, const int* Scol, const double* x,
                            double* y, cudaStream_t s, const int* done) {
    return spmv_dispatch<double>(g, Stil, Scol, x, y, s, done);
}

cudaError_t launch_spmv_pre(const Geom& g, const float* Stil, const int* Scol, const float* x,
                            float* y, cudaStream_t s, const int* done, int* stream_error) {
    if (!stream_error || ((long long)g.n_edges * 3 * g.P) % 2 != 0)
        return spmv_dispatch<float>(g, Stil, Scol, x, y, s, done);
    switch (g.P) {   // the bulk-copy pipelined kernel
        case 2: return spmv_stream_launch<6>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 3: return spmv_stream_launch<9>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 4: return spmv_stream_launch<12>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 5: return spmv_stream_launch<15>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 6: return spmv_stream_launch<18>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 7: return spmv_stream_launch<21>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 8: return spmv_stream_launch<24>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        case 9: return spmv_stream_launch<27>(g.n_edges, Stil, Scol, x, y, s, done, stream_error);
        default: return cudaErrorInvalidValue;
    }
}


cudaError_t launch_residual_norm_x2(const Geom& g, const float* Shi, const float* Slo, const int* Scol,
                                    const double* x, const double* rhs, double* w, double* scratch, double* nrm2,
                                    cudaStream_t s) {
#define CASE(P, NF)                                                                                     \
    case P: {                                                                                           \
        constexpr int EPB = 256 / NF;                                                                   \
        const int groups = (g.n_edges + EPB - 1) / EPB;                                                 \
        residual_norm_x2_kernel<NF><<<groups, 256, 0, s>>>(                                          \
            g.n_edges, Shi, Slo, Scol, x, rhs, w, scratch, nrm2);                                        \
        count_launches(1);                                                                              \
        return cudaGetLastError();                                                                      \
    }
    switch (g.P) {
        CASE(2, 6) CASE(3, 9) CASE(4, 12) CASE(5, 15) CASE(6, 18) CASE(7, 21) CASE(8, 24) CASE(9, 27)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

size_t reduction_scratch_doubles(int m, int n_edges, int P) {
    const int EPB = 256 / (3 * P);
    const size_t dots = dot_scratch_doubles(m + 2), fused = 1 + (size_t)(n_edges + EPB - 1) / EPB;
    return std::max(dots, std::max(fused, guess_scratch_doubles()));
}

}  // namespace hdgdg
