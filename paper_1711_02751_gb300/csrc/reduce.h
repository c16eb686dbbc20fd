// Deterministic grid reductions shared by the Krylov kernels: warp sums, and grid sums finished
// by the block that arrives last.
#pragma once

namespace hdgdg {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Grid reductions finish in the block that arrives last: every block writes its partial sums,
// takes a ticket, and the block holding the last ticket sums the partials in block order -- the
// same order whichever block arrives last, so results are reproducible bit for bit.  The ticket
// counter is the first word of the scratch buffer (partials follow) and is reset by that block.
__device__ inline bool last_block_arrives(unsigned* counter) {
    __shared__ unsigned s_ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
    __syncthreads();
    return s_ticket == gridDim.x - 1;
}

// s += partial[k * ld] for k = k0, k0 + stride, ... < nblk, in that order; the loads are issued
// eight at a time so that the chain of adds does not serialise them.
__device__ __forceinline__ double strided_sum(const double* partial, int k0, int stride, int nblk, size_t ld,
                                              double s) {
    for (int k = k0; k < nblk; k += 8 * stride) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = k + u * stride < nblk ? __ldcg(partial + (size_t)(k + u * stride) * ld) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    return s;
}

// out[c] = sum over blocks of partial[blk * ldp + c0 + c], c < nc: one warp per column, fixed order
__device__ inline void reduce_partials(const double* partial, int nblk, int ldp, int c0, int nc, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < nc; c += nw) {
        double s = strided_sum(partial + c0 + c, lane, 32, nblk, (size_t)ldp, 0.0);
        s = warp_sum(s);
        if (lane == 0) out[c] = s;
    }
}

}  // namespace hdgdg
