// Explicit DG residual of the nonlinear flux, stage combination, state conversion, mass.
//
// NL(q) = (F_NL(q), grad v)_K - <F*_NL . n, v>_dK   (Sec. 4.3, eq. SemiDiscretizedForm_ode)
// with F_NL = F - F_L (eq. psweFluxTensor minus eq. psweLinearFluxTensor) and the Rusanov
// flux difference F*_NL = F* - F_L* (eq. Full_russanov, eq. Linear_russanov):
//   F*_NL . n^- = {F_NL} . n^- + (tau* - tau_L*) / 2 (q^- - q^+),
//   tau* = max_pm(|u.n| + sqrt(phi)), tau_L* = max_pm sqrt(phi_B).
// Collocated GLL quadrature makes M diagonal, so M^{-1} NL at node (i, j) is
//   (2/h) [sum_a (w_a/w_i) D_ai Fx(a,j) + sum_b (w_b/w_j) D_bj Fy(i,b)]
//   - (2/h) / w_0 * (F*_NL . n) on each face through the node.
#include <atomic>

#include "internal.h"

namespace hdgdg {
namespace {

template <int P>
struct DgTile {
    static constexpr int Np = P * P;
    static constexpr int EPB = (256 / Np) > 0 ? (256 / Np) : 1;   // elements per block
};

// F_NL components along x (fx) and y (fy) for the momentum rows (the mass row is zero).
__device__ __forceinline__ void nl_flux(double ph, double U, double V, double phiB,
                                        double* fxU, double* fxV, double* fyU, double* fyV) {
    const double inv = 1.0 / (ph + phiB);
    const double half = 0.5 * ph * ph;
    const double uv = U * V * inv;
    *fxU = U * U * inv + half;
    *fxV = uv;
    *fyU = uv;
    *fyV = V * V * inv + half;
}

template <int P>
__global__ void __launch_bounds__(DgTile<P>::EPB * P * P)
dg_nl_kernel(Geom g, const double* __restrict__ q, const double* __restrict__ phiB, double scale,
             double* __restrict__ out) {
    constexpr int Np = P * P;
    constexpr int EPB = DgTile<P>::EPB;
    __shared__ double sF[EPB][4][Np];   // fxU, fxV, fyU, fyV

    const int le = threadIdx.x / Np;
    const int n = threadIdx.x % Np;
    const int e = blockIdx.x * EPB + le;
    const bool live = e < g.n_el;
    const size_t fs = (size_t)g.n_el * Np;   // field stride
    const int i = n % P, j = n / P;

    double ph = 0.0, U = 0.0, V = 0.0, pb = 1.0;
    if (live) {
        const size_t o = (size_t)e * Np + n;
        ph = q[o]; U = q[fs + o]; V = q[2 * fs + o]; pb = phiB[o];
        nl_flux(ph, U, V, pb, &sF[le][0][n], &sF[le][1][n], &sF[le][2][n], &sF[le][3][n]);
    }
    __syncthreads();
    if (!live) return;

    // volume term
    double rU = 0.0, rV = 0.0;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const double cx = g.Dhat[i * P + a];
        const double cy = g.Dhat[j * P + a];
        rU += cx * sF[le][0][j * P + a] + cy * sF[le][2][a * P + i];
        rV += cx * sF[le][1][j * P + a] + cy * sF[le][3][a * P + i];
    }
    rU *= g.two_over_h;
    rV *= g.two_over_h;
    double rph = 0.0;

    // face terms: every face through this node
    const double lift = g.two_over_h * g.inv_w0;
    const double c_own = sqrt(ph + pb);
    const double sb_own = sqrt(pb);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                        (f == 3 && j == P - 1);
        if (!on) continue;
        const int b = (f < 2) ? j : i;
        const int nb = neighbour(e, f, g.N);
        const int fo = f ^ 1;                       // opposite face of the neighbour
        const size_t o2 = (size_t)nb * Np + face_node(fo, b, P);
        const double ph2 = q[o2], U2 = q[fs + o2], V2 = q[2 * fs + o2], pb2 = phiB[o2];
        double fxU2, fxV2, fyU2, fyV2;
        nl_flux(ph2, U2, V2, pb2, &fxU2, &fxV2, &fyU2, &fyV2);
        const double sgn = (f & 1) ? 1.0 : -1.0;   // outward normal component along the face axis
        double Fo_U, Fo_V, Fn_U, Fn_V, un_o, un_n;
        if (f < 2) {
            Fo_U = sF[le][0][n]; Fo_V = sF[le][1][n]; Fn_U = fxU2; Fn_V = fxV2;
            un_o = fabs(U) / (ph + pb); un_n = fabs(U2) / (ph2 + pb2);
        } else {
            Fo_U = sF[le][2][n]; Fo_V = sF[le][3][n]; Fn_U = fyU2; Fn_V = fyV2;
            un_o = fabs(V) / (ph + pb); un_n = fabs(V2) / (ph2 + pb2);
        }
        const double tau_star = fmax(un_o + c_own, un_n + sqrt(ph2 + pb2));
        const double tau_L = fmax(sb_own, sqrt(pb2));
        const double hd = 0.5 * (tau_star - tau_L);
        const double fph = hd * (ph - ph2);
        const double fU = 0.5 * (Fo_U + Fn_U) * sgn + hd * (U - U2);
        const double fV = 0.5 * (Fo_V + Fn_V) * sgn + hd * (V - V2);
        rph -= lift * fph;
        rU -= lift * fU;
        rV -= lift * fV;
    }
    const size_t o = (size_t)e * Np + n;
    out[o] = scale * rph;
    out[fs + o] = scale * rU;
    out[2 * fs + o] = scale * rV;
}

__global__ void combine_kernel(size_t n, const double* __restrict__ base, CombineTerms t,
                               double* out, unsigned* nonfinite) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        double acc = base[idx];
        for (int k = 0; k < t.n; ++k) acc += t.c[k] * t.X[k][idx];
        out[idx] = acc;
        if (nonfinite && !isfinite(acc)) *nonfinite = 1u;
    }
}

__global__ void user_to_state_kernel(Geom g, const double* __restrict__ h, const double* __restrict__ hu,
                                     const double* __restrict__ hv, const double* __restrict__ phiB,
                                     double gacc, double* __restrict__ q, unsigned* bad) {
    const size_t n = (size_t)g.n_el * g.Np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const double phi = gacc * h[idx];
        const double ph = phi - phiB[idx];
        const double U = gacc * hu[idx], V = gacc * hv[idx];
        if (!isfinite(phi) || !isfinite(U) || !isfinite(V) || !(phi > 0.0)) *bad = 1u;
        q[idx] = ph;
        q[n + idx] = U;
        q[2 * n + idx] = V;
    }
}

__global__ void state_to_user_kernel(Geom g, const double* __restrict__ q, const double* __restrict__ phiB,
                                     double gacc, double* __restrict__ h, double* __restrict__ hu,
                                     double* __restrict__ hv) {
    const size_t n = (size_t)g.n_el * g.Np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        h[idx] = (q[idx] + phiB[idx]) / gacc;
        hu[idx] = q[n + idx] / gacc;
        hv[idx] = q[2 * n + idx] / gacc;
    }
}

constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__global__ void mass_partial_kernel(Geom g, const double* __restrict__ q, double* partial) {
    __shared__ double sh[32];
    const size_t n = (size_t)g.n_el * g.Np;
    double acc = 0.0;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int node = (int)(idx % g.Np);
        acc += g.w[node % g.P] * g.w[node / g.P] * q[idx];
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void mass_final_kernel(const double* partial, int nb, double J, double* out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += partial[k];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = J * acc;
}

template <int P>
cudaError_t dg_nl_launch(const Geom& g, const double* q, const double* phiB, double scale,
                         double* out, cudaStream_t s) {
    constexpr int EPB = DgTile<P>::EPB;
    const int blocks = (g.n_el + EPB - 1) / EPB;
    dg_nl_kernel<P><<<blocks, EPB * P * P, 0, s>>>(g, q, phiB, scale, out);
    count_launches(1);
    return cudaGetLastError();
}

int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return b > 0 ? (int)b : 1;
}

}  // namespace

namespace {
std::atomic<long long> g_launches{0};
}

long long launches_total() { return g_launches.load(); }
void count_launches(int n) { g_launches.fetch_add(n); }

cudaError_t launch_dg_nl(const Geom& g, const double* q, const double* phiB, double scale,
                         double* out, cudaStream_t s) {
    switch (g.P) {
        case 2: return dg_nl_launch<2>(g, q, phiB, scale, out, s);
        case 3: return dg_nl_launch<3>(g, q, phiB, scale, out, s);
        case 4: return dg_nl_launch<4>(g, q, phiB, scale, out, s);
        case 5: return dg_nl_launch<5>(g, q, phiB, scale, out, s);
        case 6: return dg_nl_launch<6>(g, q, phiB, scale, out, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_combine(size_t n, const double* base, const CombineTerms& t, double* out,
                           unsigned* nonfinite_flag, cudaStream_t s) {
    combine_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, base, t, out, nonfinite_flag);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_user_to_state(const Geom& g, const double* h, const double* hu, const double* hv,
                                 const double* phiB, double gacc, double* q, unsigned* bad,
                                 cudaStream_t s) {
    const size_t n = (size_t)g.n_el * g.Np;
    user_to_state_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, h, hu, hv, phiB, gacc, q, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_state_to_user(const Geom& g, const double* q, const double* phiB, double gacc,
                                 double* h, double* hu, double* hv, cudaStream_t s) {
    const size_t n = (size_t)g.n_el * g.Np;
    state_to_user_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, q, phiB, gacc, h, hu, hv);
    count_launches(1);
    return cudaGetLastError();
}

size_t mass_scratch_doubles() { return kRedBlocks; }

cudaError_t launch_mass(const Geom& g, const double* q, double* scratch, double* out, cudaStream_t s) {
    mass_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(g, q, scratch);
    count_launches(1);
    mass_final_kernel<<<1, kRedThreads, 0, s>>>(scratch, kRedBlocks, g.J, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hdgdg
