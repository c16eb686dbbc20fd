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
// tau_L* = max_pm sqrt(phi_B) is the per-edge-node tau_hat the library precomputes.
#include <atomic>

#include <cuda_bf16.h>

#include "ens.h"
#include "fastcvt.h"
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace hdgdg {
namespace {

template <int P>
struct DgTile {
    static constexpr int Np = P * P;
    static constexpr int EPB = (256 / Np) > 0 ? (256 / Np) : 1;   // elements per block
};

// An input of the residual in the arithmetic type; BF: rounded to BF16 first (8 significant bits,
// nearest even), the BF16-input variant of the mixed form.  An input already stored in FP32 (the
// mixed form's FP32 copies, rounded the same way) passes as it is.
template <typename Tc, bool BF>
__device__ __forceinline__ Tc dg_in(double v) {
    if constexpr (BF) return __bfloat162float(__float2bfloat16_rn(f64_to_f32(v)));
    else return from_f64<Tc>(v);
}
template <typename Tc, bool BF>
__device__ __forceinline__ Tc dg_in(float v) {
    static_assert(sizeof(Tc) == 4 && !BF, "FP32 inputs feed the FP32 residual");
    return v;
}

// A stored value as the local type TV of the face pass (double, or float for FP32 inputs).
template <typename TV, typename TI>
__device__ __forceinline__ TV as_tv(TI v) {
    if constexpr (sizeof(TV) == sizeof(TI)) return v;
    else if constexpr (sizeof(TV) == 4) return f64_to_f32(v);
    else return (double)v;
}

// F_NL components along x (fx) and y (fy) for the momentum rows (the mass row is zero).
template <typename Tc>
__device__ __forceinline__ void nl_flux(Tc ph, Tc U, Tc V, Tc phiB, Tc* fxU, Tc* fxV, Tc* fyU, Tc* fyV) {
    const Tc inv = Tc(1) / (ph + phiB);
    const Tc half = Tc(0.5) * ph * ph;
    const Tc uv = U * V * inv;
    *fxU = U * U * inv + half;
    *fxV = uv;
    *fyU = uv;
    *fyV = V * V * inv + half;
}

// Face pass: the Rusanov flux difference F*_NL . n through every edge node, computed once per
// node (so the two elements see exactly opposite values) and stored as the flux along the
// edge's +x / +y normal: fface[edge][c][b].  One thread per (edge, b).
//   FULL = true: the Rusanov flux F* . n of the whole flux F = F_NL + F_L (eq. Full_russanov),
//   the residual of the explicit RK DG scheme the paper compares with.
//   Tc: arithmetic type (double; float for the mixed form's residual), storage stays FP64.
// A32: phi_B, tau and the face fluxes stored in FP32 (the mixed form's copies; Tc = float);
// TQ: the type the state q is stored in (FP32: the recovery's FP32 stage values).
template <int P, bool FULL, typename Tc, bool BF = false, typename TQ = double, bool A32 = false>
__device__ __forceinline__ void dg_face_body(int bid, const Geom& g, const TQ* __restrict__ q,
                                             const std::conditional_t<A32, float, double>* __restrict__ phiB,
                                             const std::conditional_t<A32, float, double>* __restrict__ tau_edge,
                                             std::conditional_t<A32, float, double>* __restrict__ fface,
                                             double t_bc) {
    using TV = std::conditional_t<A32, float, double>;   // the node values as the pass holds them
    constexpr int Np = P * P;
    const int t = bid * 256 + threadIdx.x;
    if (t >= g.n_edges * P) return;
    const int r = t / P, b = t % P;
    int em, fm, ep, fp;
    edge_sides(r, g, &em, &fm, &ep, &fp);
    const size_t fs = (size_t)g.n_el * Np;
    const bool xedge = fm == 1;
    TV phm, Um, Vm, pbm, php, Up, Vp, pbp;
    if (em >= 0) {
        const size_t om = (size_t)em * Np + face_node(fm, b, P);
        phm = as_tv<TV>(q[om]); Um = as_tv<TV>(q[fs + om]); Vm = as_tv<TV>(q[2 * fs + om]); pbm = phiB[om];
    }
    if (ep >= 0) {
        const size_t op = (size_t)ep * Np + face_node(fp, b, P);
        php = as_tv<TV>(q[op]); Up = as_tv<TV>(q[fs + op]); Vp = as_tv<TV>(q[2 * fs + op]); pbp = phiB[op];
    }
    if (g.dirichlet && (em < 0 || ep < 0)) {
        // Dirichlet boundary: the other side is the prescribed exact state at the node
        double x, y;
        face_node_xy(g, em >= 0 ? em : ep, em >= 0 ? fm : fp, b, &x, &y);
        double ph, U, V;
        vortex_state(g, x, y, t_bc * dt_factor(g, em >= 0 ? em : ep), &ph, &U, &V);
        if (em < 0) { phm = as_tv<TV>(ph); Um = as_tv<TV>(U); Vm = as_tv<TV>(V); pbm = pbp; }
        else { php = as_tv<TV>(ph); Up = as_tv<TV>(U); Vp = as_tv<TV>(V); pbp = pbm; }
    } else {
        // a wall edge sees the mirror state of its one element (eq. reflection): same phi and
        // tangential momentum, opposite normal momentum
        if (em < 0) { phm = php; pbm = pbp; Um = xedge ? -Up : Up; Vm = xedge ? Vp : -Vp; }
        if (ep < 0) { php = phm; pbp = pbm; Up = xedge ? -Um : Um; Vp = xedge ? Vm : -Vm; }
    }
    // (conversions to the arithmetic type on the integer pipes, fastcvt.h)
    const Tc pm = dg_in<Tc, BF>(phm), pp = dg_in<Tc, BF>(php);
    const Tc Phm = pm + dg_in<Tc, BF>(pbm), Php = pp + dg_in<Tc, BF>(pbp);
    const Tc im = Tc(1) / Phm, ip = Tc(1) / Php;
    // normal (n) and tangential (t) momentum components along this edge's +axis
    const Tc Unm = dg_in<Tc, BF>(xedge ? Um : Vm), Utm = dg_in<Tc, BF>(xedge ? Vm : Um);
    const Tc Unp = dg_in<Tc, BF>(xedge ? Up : Vp), Utp = dg_in<Tc, BF>(xedge ? Vp : Up);
    // F_NL . n: (0, Un Un / phi + phi_eta^2 / 2, Un Ut / phi) in (normal, tangential) order
    Tc Fnm = Unm * Unm * im + Tc(0.5) * pm * pm, Ftm = Unm * Utm * im;
    Tc Fnp = Unp * Unp * ip + Tc(0.5) * pp * pp, Ftp = Unp * Utp * ip;
    const Tc tau_star = fmax(fabs(Unm) * im + sqrt(Phm), fabs(Unp) * ip + sqrt(Php));
    Tc hd, fph;
    if (FULL) {   // add F_L . n = (U_n, phi_eta phi_B, 0)
        Fnm += pm * dg_in<Tc, false>(pbm);
        Fnp += pp * dg_in<Tc, false>(pbp);
        hd = Tc(0.5) * tau_star;
        fph = Tc(0.5) * (Unm + Unp) + hd * (pm - pp);
    } else {
        hd = Tc(0.5) * (tau_star - dg_in<Tc, BF>(tau_edge[(size_t)r * P + b]));
        fph = hd * (pm - pp);
    }
    const Tc fn = Tc(0.5) * (Fnm + Fnp) + hd * (Unm - Unp);
    const Tc ft = Tc(0.5) * (Ftm + Ftp) + hd * (Utm - Utp);
    TV* out = fface + (size_t)r * 3 * P;
    if constexpr (A32) {   // FP32 storage: the values the FP64 storage's round trip gives back
        out[b] = fph;
        out[(xedge ? 1 : 2) * P + b] = fn;
        out[(xedge ? 2 : 1) * P + b] = ft;
    } else {
        out[b] = to_f64(fph);
        out[(xedge ? 1 : 2) * P + b] = to_f64(fn);
        out[(xedge ? 2 : 1) * P + b] = to_f64(ft);
    }
}

template <int P, bool FULL, typename Tc, bool BF = false, typename TQ = double, bool A32 = false>
__global__ void __launch_bounds__(256)
dg_face_kernel(Geom g, const TQ* __restrict__ q, const std::conditional_t<A32, float, double>* __restrict__ phiB,
               const std::conditional_t<A32, float, double>* __restrict__ tau_edge,
               std::conditional_t<A32, float, double>* __restrict__ fface, double t_bc) {
    dg_face_body<P, FULL, Tc, BF, TQ, A32>(blockIdx.x, g, q, phiB, tau_edge, fface, t_bc);
}

// The step's final update at node o (field stride fs) with this pass's residual v as term
// fin.slot: every other term's loads issued before the sums, each field's terms added in their
// order as combine_kernel adds them.
__device__ __forceinline__ void dg_final_update(const FinalSource& fin, size_t o, size_t fs, const double v[3]) {
    double acc[3], x[kFinalTerms][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = fin.base[o + c * fs];
#pragma unroll
    for (int k = 0; k < kFinalTerms; ++k)   // constant indices keep the terms in the parameter bank
        if (k < fin.t.n && k != fin.slot) {
#pragma unroll
            for (int c = 0; c < 3; ++c) x[k][c] = fin.t.X[k][o + c * fs];
        }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int k = 0; k < kFinalTerms; ++k)
            if (k < fin.t.n) acc[c] += fin.t.c[k] * (k == fin.slot ? v[c] : x[k][c]);
        fin.qn[o + c * fs] = acc[c];
        bad |= !isfinite(acc[c]);
    }
    if (bad && fin.nonfinite) *fin.nonfinite = 1u;
}

// Element pass: volume term from the nodal F_NL (shared memory), minus the lifted face fluxes.
// FULL = true: the whole flux F and the source s = (0, phi_eta d_x phi_B, phi_eta d_y phi_B).
template <int P, bool FULL, typename Tc, bool BF = false, typename TQ = double, bool A32 = false, bool FIN = false>
__device__ __forceinline__ void dg_volume_body(int bid, const Geom& g, const TQ* __restrict__ q,
                                               const std::conditional_t<A32, float, double>* __restrict__ phiB,
                                               const std::conditional_t<A32, float, double>* __restrict__ fface,
                                               double scale, double* __restrict__ out,
                                               const FinalSource& fin = FinalSource{}) {
    constexpr int Np = P * P;
    constexpr int EPB = DgTile<P>::EPB;
    // fxU, fxV, fyU, fyV (and, FULL: U, V, phi_B) per element, each element's row padded by one
    // word so that the two or more elements a warp covers fall in different banks
    __shared__ Tc sFr[EPB][4 * Np + 1];
    __shared__ Tc sMr[FULL ? EPB : 1][3 * Np + 1];
    // the derivative matrices, read below with a thread-dependent row: from shared memory, since
    // the kernel-parameter (constant) bank serialises a warp's loads of different addresses
    __shared__ Tc sDh[Np], sD[Np];
    if (threadIdx.x < Np) {
        sDh[threadIdx.x] = from_f64<Tc>(g.Dhat[threadIdx.x]);
        sD[threadIdx.x] = from_f64<Tc>(g.D[threadIdx.x]);
    }

    const int le = threadIdx.x / Np;
    const int n = threadIdx.x % Np;
    const int e = bid * EPB + le;
    const bool live = le < EPB && e < g.n_el;
    const size_t fs = (size_t)g.n_el * Np;
    const int i = n % P, j = n / P;

    Tc ph_own = Tc(0);
    if (live) {
        const size_t o = (size_t)e * Np + n;
        const Tc ph = dg_in<Tc, BF>(q[o]), U = dg_in<Tc, BF>(q[fs + o]), V = dg_in<Tc, BF>(q[2 * fs + o]),
                 pb = dg_in<Tc, BF>(phiB[o]);
        nl_flux<Tc>(ph, U, V, pb, &sFr[le][0 * Np + n], &sFr[le][1 * Np + n], &sFr[le][2 * Np + n], &sFr[le][3 * Np + n]);
        if (FULL) {
            sFr[le][0 * Np + n] += ph * pb;
            sFr[le][3 * Np + n] += ph * pb;
            sMr[FULL ? le : 0][0 * Np + n] = U;
            sMr[FULL ? le : 0][1 * Np + n] = V;
            sMr[FULL ? le : 0][2 * Np + n] = pb;
            ph_own = ph;
        }
    }
    __syncthreads();
    if (!live) return;

    Tc rU = Tc(0), rV = Tc(0), rph = Tc(0);
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const Tc cx = sDh[i * P + a];
        const Tc cy = sDh[j * P + a];
        rU += cx * sFr[le][0 * Np + j * P + a] + cy * sFr[le][2 * Np + a * P + i];
        rV += cx * sFr[le][1 * Np + j * P + a] + cy * sFr[le][3 * Np + a * P + i];
        if (FULL) rph += cx * sMr[le][0 * Np + j * P + a] + cy * sMr[le][1 * Np + a * P + i];
    }
    const Tc th = from_f64<Tc>(g.two_over_h);
    rU *= th;
    rV *= th;
    rph *= th;
    if (FULL) {   // source phi_eta grad phi_B with the nodal derivative of phi_B
        Tc dBx = Tc(0), dBy = Tc(0);
#pragma unroll
        for (int a = 0; a < P; ++a) {
            dBx += sD[i * P + a] * sMr[le][2 * Np + j * P + a];
            dBy += sD[j * P + a] * sMr[le][2 * Np + a * P + i];
        }
        rU += ph_own * th * dBx;
        rV += ph_own * th * dBy;
    }
    const Tc lift = from_f64<Tc>(g.two_over_h * g.inv_w0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                        (f == 3 && j == P - 1);
        if (!on) continue;
        const int b = (f < 2) ? j : i;
        const auto* fl = fface + (size_t)edge_of_face(e, f, g) * 3 * P;
        const Tc sgn = (f & 1) ? lift : -lift;   // outward normal is + on faces 1, 3
        rph -= sgn * dg_in<Tc, false>(fl[b]);
        rU -= sgn * dg_in<Tc, false>(fl[P + b]);
        rV -= sgn * dg_in<Tc, false>(fl[2 * P + b]);
    }
    const size_t o = (size_t)e * Np + n;
    const double sc = scale * dt_factor(g, e);   // this instance's time step
    const double v[3] = {sc * to_f64(rph), sc * to_f64(rU), sc * to_f64(rV)};
    if constexpr (FIN) {   // its own instance: the other passes keep their registers
        dg_final_update(fin, o, fs, v);
        return;
    }
    out[o] = v[0];
    out[fs + o] = v[1];
    out[2 * fs + o] = v[2];
}

template <int P, bool FULL, typename Tc, bool BF = false, typename TQ = double, bool A32 = false, bool FIN = false>
__global__ void __launch_bounds__(DgTile<P>::EPB * P * P)
dg_volume_kernel(Geom g, const TQ* __restrict__ q, const std::conditional_t<A32, float, double>* __restrict__ phiB,
                 const std::conditional_t<A32, float, double>* __restrict__ fface, double scale,
                 double* __restrict__ out, FinalSource fin) {
    dg_volume_body<P, FULL, Tc, BF, TQ, A32, FIN>(blockIdx.x, g, q, phiB, fface, scale, out, fin);
}

// One instance per term count NT (0..10), the terms indexed by constants.  Each thread takes U
// lanes of L entries (L = 2: 16-byte loads, every vector 16-byte aligned and n even) a grid apart
// per pass and issues all their loads before the first sum; each entry's terms are added in their
// order, so the lane width changes no result.
template <int L>
__device__ __forceinline__ void load_l(const double* __restrict__ p, size_t i, double* v) {
    if constexpr (L == 2) {
        const double2 q = reinterpret_cast<const double2*>(p)[i];
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = p[i];
    }
}

template <int NT, int L>
__global__ void combine_kernel(size_t n, const double* __restrict__ base, CombineTerms t,
                               double* out, unsigned* nonfinite) {
    constexpr int U = NT <= 2 ? 4 : 2;
    const size_t stride = (size_t)gridDim.x * blockDim.x, nl = n / L;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < nl; i0 += U * stride) {
        double acc[U][L], xv[U][NT > 0 ? NT : 1][L];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t il = i0 + u * stride;
            if (il < nl) {
                load_l<L>(base, il, acc[u]);
#pragma unroll
                for (int k = 0; k < NT; ++k) load_l<L>(t.X[k], il, xv[u][k]);
            }
        }
        bool bad = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t il = i0 + u * stride;
            if (il >= nl) continue;
#pragma unroll
            for (int l = 0; l < L; ++l) {
#pragma unroll
                for (int k = 0; k < NT; ++k) acc[u][l] += t.c[k] * xv[u][k][l];
                out[il * L + l] = acc[u][l];
                bad |= !isfinite(acc[u][l]);
            }
        }
        if (nonfinite && bad) *nonfinite = 1u;
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

template <int P, bool FULL, typename Tc = double, bool BF = false>
cudaError_t dg_launch(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                      double scale, double* fface, double* out, cudaStream_t s, double t) {
    constexpr int EPB = DgTile<P>::EPB;
    const int nf = g.n_edges * P;
    dg_face_kernel<P, FULL, Tc, BF><<<(nf + 255) / 256, 256, 0, s>>>(g, q, phiB, tau_edge, fface, t);
    count_launches(1);
    dg_volume_kernel<P, FULL, Tc, BF><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(g, q, phiB, fface, scale, out,
                                                                                      FinalSource{});
    count_launches(1);
    return cudaGetLastError();
}

// The mixed form's residual on FP32 copies: phi_B, tau and the face fluxes in FP32, the state
// in FP32 (q32, the recovery's FP32 stage values) or FP64 (q64, the step's start).
template <int P>
cudaError_t dg_launch_f32io(const Geom& g, const double* q64, const float* q32, const float* phiB,
                            const float* tau_edge, double scale, float* fface, double* out, cudaStream_t s,
                            double t, const FinalSource& fin) {
    constexpr int EPB = DgTile<P>::EPB;
    const int nf = g.n_edges * P;
    const int gf = (nf + 255) / 256, gv = (g.n_el + EPB - 1) / EPB, tv = EPB * P * P;
    if (q32) {
        dg_face_kernel<P, false, float, false, float, true><<<gf, 256, 0, s>>>(g, q32, phiB, tau_edge, fface, t);
        if (fin.base)
            dg_volume_kernel<P, false, float, false, float, true, true><<<gv, tv, 0, s>>>(g, q32, phiB, fface, scale,
                                                                                        out, fin);
        else
            dg_volume_kernel<P, false, float, false, float, true><<<gv, tv, 0, s>>>(g, q32, phiB, fface, scale, out,
                                                                                  fin);
    } else {
        dg_face_kernel<P, false, float, false, double, true><<<gf, 256, 0, s>>>(g, q64, phiB, tau_edge, fface, t);
        dg_volume_kernel<P, false, float, false, double, true><<<gv, tv, 0, s>>>(g, q64, phiB, fface, scale, out,
                                                                                 fin);
    }
    count_launches(2);
    return cudaGetLastError();
}

int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return b > 0 ? (int)b : 1;
}

// ---- ensembles: every group's face and element passes in one persistent launch each ---------------
template <int P>
__device__ __forceinline__ void ens_face_item(const EnsGroup& G, int bid, const double* q, double* fface) {
    dg_face_body<P, false, float>(bid, G.g, q + G.off3, G.phiB, G.tau, fface + G.offt, 0.0);
}

__global__ void __launch_bounds__(256) ens_dg_face_kernel(EnsTable t, const double* __restrict__ q,
                                                          double* __restrict__ fface) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        switch (G.g.P) {
            case 3: ens_face_item<3>(G, bid, q, fface); break;
            case 4: ens_face_item<4>(G, bid, q, fface); break;
            case 5: ens_face_item<5>(G, bid, q, fface); break;
            default: break;
        }
    });
}

__global__ void __launch_bounds__(256) ens_dg_volume_kernel(EnsTable t, const double* __restrict__ q,
                                                            const double* __restrict__ fface, double* __restrict__ out) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        switch (G.g.P) {
            case 3: dg_volume_body<3, false, float>(bid, G.g, q + G.off3, G.phiB, fface + G.offt, G.dt, out + G.off3); break;
            case 4: dg_volume_body<4, false, float>(bid, G.g, q + G.off3, G.phiB, fface + G.offt, G.dt, out + G.off3); break;
            case 5: dg_volume_body<5, false, float>(bid, G.g, q + G.off3, G.phiB, fface + G.offt, G.dt, out + G.off3); break;
            default: break;
        }
    });
}

}  // namespace

cudaError_t launch_ens_dg_nl_f32(const EnsHost& E, const double* q, double* fface, double* out, cudaStream_t s) {
    const EnsTable tf = ens_table(E, [](const EnsGroup& G) { return (G.g.n_edges * G.g.P + 255) / 256; });
    const EnsTable tv = ens_table(E, [](const EnsGroup& G) {
        const int epb = 256 / G.g.Np;
        return (G.g.n_el + epb - 1) / epb;
    });
    ens_dg_face_kernel<<<ens_grid(ens_dg_face_kernel, tf.start[tf.ngroups]), 256, 0, s>>>(tf, q, fface);
    ens_dg_volume_kernel<<<ens_grid(ens_dg_volume_kernel, tv.start[tv.ngroups]), 256, 0, s>>>(tv, q, fface, out);
    count_launches(2);
    return cudaGetLastError();
}

namespace {
std::atomic<long long> g_launches{0};
}

long long launches_total() { return g_launches.load(); }
void count_launches(int n) { g_launches.fetch_add(n); }

cudaError_t launch_dg_nl(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                         double scale, double* fface, double* out, cudaStream_t s, double t) {
    switch (g.P) {
        case 2: return dg_launch<2, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 3: return dg_launch<3, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 4: return dg_launch<4, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 5: return dg_launch<5, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 6: return dg_launch<6, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 7: return dg_launch<7, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 8: return dg_launch<8, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 9: return dg_launch<9, false>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dg_nl_f32io(const Geom& g, const double* q64, const float* q32, const float* phiB32,
                               const float* tau32, double scale, float* fface32, double* out, cudaStream_t s,
                               double t, const FinalSource* fin) {
    const FinalSource none{};
    if (fin && fin->base && (fin->t.n < 1 || fin->t.n > kFinalTerms || fin->slot < 0 || fin->slot >= fin->t.n ||
                             !fin->qn))
        return cudaErrorInvalidValue;
    const FinalSource& f = fin ? *fin : none;
    switch (g.P) {
#define CASE(P) \
    case P: return dg_launch_f32io<P>(g, q64, q32, phiB32, tau32, scale, fface32, out, s, t, f);
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dg_nl_f32(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                             double scale, double* fface, double* out, cudaStream_t s, double t) {
    switch (g.P) {
        case 2: return dg_launch<2, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 3: return dg_launch<3, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 4: return dg_launch<4, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 5: return dg_launch<5, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 6: return dg_launch<6, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 7: return dg_launch<7, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 8: return dg_launch<8, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 9: return dg_launch<9, false, float>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dg_nl_bf16(const Geom& g, const double* q, const double* phiB, const double* tau_edge,
                              double scale, double* fface, double* out, cudaStream_t s, double t) {
    switch (g.P) {
        case 2: return dg_launch<2, false, float, true>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 3: return dg_launch<3, false, float, true>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 4: return dg_launch<4, false, float, true>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        case 5: return dg_launch<5, false, float, true>(g, q, phiB, tau_edge, scale, fface, out, s, t);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dg_full(const Geom& g, const double* q, const double* phiB, double scale,
                           double* fface, double* out, cudaStream_t s, double t) {
    switch (g.P) {
        case 2: return dg_launch<2, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 3: return dg_launch<3, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 4: return dg_launch<4, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 5: return dg_launch<5, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 6: return dg_launch<6, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 7: return dg_launch<7, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 8: return dg_launch<8, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        case 9: return dg_launch<9, true>(g, q, phiB, nullptr, scale, fface, out, s, t);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_combine(size_t n, const double* base, const CombineTerms& t, double* out,
                           unsigned* nonfinite_flag, cudaStream_t s) {
    if (t.n < 0 || t.n > 10) return cudaErrorInvalidValue;
    bool l2 = n % 2 == 0 && reinterpret_cast<uintptr_t>(base) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0;
    for (int k = 0; k < t.n; ++k) l2 = l2 && reinterpret_cast<uintptr_t>(t.X[k]) % 16 == 0;
    const int grid = grid_for(l2 ? n / 2 : n, 256);
    switch (t.n) {
#define CASE(K)                                                                                 \
    case K:                                                                                     \
        if (l2) combine_kernel<K, 2><<<grid, 256, 0, s>>>(n, base, t, out, nonfinite_flag); \
        else combine_kernel<K, 1><<<grid, 256, 0, s>>>(n, base, t, out, nonfinite_flag);     \
        break;
        CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
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
