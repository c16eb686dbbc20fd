// Work-list walk of the ensemble launches (see EnsTable in internal.h): a persistent grid of
// 256-thread blocks takes the items (group, block of the group) in turn.  Every item's body is a
// lone kernel's block body run with that group's geometry and slices; a barrier separates items,
// since consecutive items of one block reuse its shared memory.
#pragma once

#include <algorithm>

#include "internal.h"

namespace hdgdg {

template <class F>
__device__ __forceinline__ void ens_walk(const EnsTable& t, F&& body) {
    const int total = t.start[t.ngroups];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int gi = 0;
        while (item >= t.start[gi + 1]) ++gi;
        body(t.grp[gi], item - t.start[gi]);
        __syncthreads();
    }
}

// The launch table for a kind of work: blocks(group) blocks for each group.
template <class Blocks>
EnsTable ens_table(const EnsHost& E, Blocks blocks) {
    EnsTable t{};
    t.grp = E.d_grp;
    t.ngroups = E.ngroups;
    t.start[0] = 0;
    for (int i = 0; i < E.ngroups; ++i) t.start[i + 1] = t.start[i] + blocks(E.h[i]);
    return t;
}

// Persistent grid: as many 256-thread blocks as fit on the device at once, at most one per item.
template <class K>
int ens_grid(K kernel, int items) {
    static int per_sm = 0, sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 256, 0) != cudaSuccess || nb <= 0) nb = 1;
    per_sm = nb;
    const int grid = per_sm * sms;
    return std::max(1, std::min(items, grid));
}

}  // namespace hdgdg
