// Allocation-free variant of the mass reduction behind hdgdg_get_stats.
//
// Some callers cannot allocate device memory at the point where they need the mass of a
// state: code that runs inside another framework's fixed memory pool, a real-time loop that
// must not enter the CUDA allocator, or a host callback that may not call cudaMalloc.  This
// entry point takes the state and the output from the caller and keeps its own partial sums
// in a fixed-size array in the library's static device memory, which every GPU that loads
// the library holds until the process exits.
#include <cmath>

#include "hdgdg.h"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxElements = 1 << 20;   // 8 MiB of per-element partial sums per device

// Per-element partial masses of the current call.  Shared by every call on a device: calls
// that overlap on the GPU race on it.
static __device__ __align__(256) double g_elem_mass[kNoAllocMaxElements];

// m_e = sum_ij w_i w_j phi_eta(e, i, j), one thread per element.
__global__ void elem_mass_kernel(int n_el, int P, hdgdg::Geom g, const double* __restrict__ phi,
                                 double* __restrict__ part) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const double* p = phi + (size_t)e * P * P;
    double acc = 0.0;
    for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) acc += g.w[i] * g.w[j] * p[j * P + i];
    part[e] = acc;
}

// out = J * sum_e m_e: one block, fixed order (strided per-thread sums, then a tree).
__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double J, double* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = J * sh[0];
}

// Device address of the static scratch in the current context.  Looked up on every call (the
// lookup allocates nothing and is cheap), so a context that was torn down and created again,
// which may place the module's static memory elsewhere, never sees a stale address.
cudaError_t scratch_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_elem_mass);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" hdgdg_status hdgdg_mass_noalloc(int n_side, int degree_k, double length, const double* d_phi_eta,
                                           double* d_mass, void* cuda_stream) {
    if (n_side < 1 || degree_k < 1 || degree_k > hdgdg::kMaxP - 1 || !d_phi_eta || !d_mass ||
        !std::isfinite(length))
        return HDGDG_EINVAL;
    const long long n_el = (long long)n_side * n_side;
    if (n_el > kNoAllocMaxElements) return HDGDG_EINVAL;   // beyond the static scratch
    hdgdg::Geom g = hdgdg::host_geom(n_side, degree_k);
    const double L = length > 0.0 ? length : 1.0;
    const double J = 0.25 * (L / n_side) * (L / n_side);   // element Jacobian (h/2)^2, h = L/N
    double* part = nullptr;
    if (scratch_address(&part) != cudaSuccess) return HDGDG_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int threads = 256;
    elem_mass_kernel<<<(int)((n_el + threads - 1) / threads), threads, 0, s>>>((int)n_el, g.P, g, d_phi_eta, part);
    sum_partials_kernel<<<1, 256, 0, s>>>(part, (int)n_el, J, d_mass);
    hdgdg::count_launches(2);
    return cudaGetLastError() == cudaSuccess ? HDGDG_OK : HDGDG_ECUDA;
}
