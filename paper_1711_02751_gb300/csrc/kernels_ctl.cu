// Device-side control of the trace solve inside a whole-step CUDA graph.
//
// A time step of Algorithm 1 is captured once per pointer configuration and replayed as ONE
// graph: each implicit stage's trace solve chooses its initial guess, runs its restart cycles
// inside a conditional (while) node and records its counters without returning to the host.
// The decisions the host driver takes between restart cycles -- the extrapolation order whose
// residual is smallest, the stop tests on the true residual, the iteration cap -- are taken here
// by one-thread kernels, in the same order and with the same arithmetic, so a replayed step
// gives the same numbers as the host-driven one.
#include "internal.h"

namespace hdgdg {
namespace {

// Begin a solve: ||g||^2 = cand[0], the candidates' squared residual norms cand[1..avail];
// chooses the start (zero or the extrapolation order with the smallest finite residual), sets the
// absolute tolerance and the GMRES control block, and writes the start's squared residual norm.
__device__ __forceinline__ void solve_begin_body(const double* __restrict__ cand, int avail, double rtol,
                                                 double inner_rel, int maxit, GmresCtl* ctl, SolveCtl* sc,
                                                 StepStats* ss, double* nrm2) {
    const double bn2 = cand[0];
    sc->active = 0;
    sc->guess = 0;
    sc->bnorm = 0.0;
    sc->tol = 0.0;
    ctl->tol_abs = 0.0;
    ctl->inner_rel = inner_rel;
    ctl->maxit = maxit;
    ctl->total = 0;
    ctl->status = 0;
    if (!isfinite(bn2)) {
        ss->nonfinite = 1u;
        *nrm2 = 0.0;
        return;
    }
    if (bn2 == 0.0) {   // g = 0: qhat = 0
        *nrm2 = 0.0;
        return;
    }
    int guess = 0;
    for (int q = 1; q <= avail; ++q)
        if (isfinite(cand[q]) && cand[q] < cand[guess]) guess = q;
    sc->active = 1;
    sc->guess = guess;
    sc->bnorm = sqrt(bn2);
    sc->tol = rtol * sc->bnorm;
    ctl->tol_abs = sc->tol;
    ss->last_guess = guess;
    *nrm2 = cand[guess];
}

__global__ void solve_begin_kernel(const double* __restrict__ cand, int avail, double rtol, double inner_rel,
                                   int maxit, GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double* nrm2) {
    solve_begin_body(cand, avail, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
}

// the same with the number of candidates read from the step's history table
__global__ void solve_begin_dev_kernel(const double* __restrict__ cand, const DevHist* __restrict__ dh, double rtol,
                                       double inner_rel, int maxit, GmresCtl* ctl, SolveCtl* sc, StepStats* ss,
                                       double* nrm2) {
    solve_begin_body(cand, dh->avail, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
}

// x~ = x_{n-1} + sum_j (c_qj - [j = 0]) x_{n-1-j} and w = g - sum_j c_qj S~x_{n-1-j} for the chosen
// order q (the host driver's two combinations, term for term); q = 0: x~ = 0, w = g.  One loop
// per order, its terms indexed by constants.
template <int Q>
__device__ __forceinline__ void guess_apply_order(size_t n, const double* __restrict__ g, const GuessHistory& h,
                                                  double* __restrict__ xt, double* __restrict__ w) {
    constexpr int U = 2;   // entries a grid apart per pass, every load issued before the sums
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        if constexpr (Q == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t idx = i0 + u * stride;
                if (idx < n) {
                    xt[idx] = 0.0;
                    w[idx] = g[idx];
                }
            }
        } else {
            double xv[U][Q], yv[U][Q], gv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t idx = i0 + u * stride;
                if (idx < n) {
                    gv[u] = g[idx];
#pragma unroll
                    for (int j = 0; j < Q; ++j) {
                        xv[u][j] = h.x[j][idx];
                        yv[u][j] = h.y[j][idx];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t idx = i0 + u * stride;
                if (idx >= n) continue;
                double ax = xv[u][0];
#pragma unroll
                for (int j = 0; j < Q; ++j) ax += (h.c[Q][j] - (j == 0 ? 1.0 : 0.0)) * xv[u][j];
                double aw = gv[u];
#pragma unroll
                for (int j = 0; j < Q; ++j) aw += (-h.c[Q][j]) * yv[u][j];
                xt[idx] = ax;
                w[idx] = aw;
            }
        }
    }
}

__device__ __forceinline__ void guess_apply_body(size_t n, const double* __restrict__ g, const GuessHistory& h,
                                                 const SolveCtl* __restrict__ sc, double* __restrict__ xt,
                                                 double* __restrict__ w) {
    switch (sc->active ? sc->guess : 0) {
        case 1: return guess_apply_order<1>(n, g, h, xt, w);
        case 2: return guess_apply_order<2>(n, g, h, xt, w);
        case 3: return guess_apply_order<3>(n, g, h, xt, w);
        case 4: return guess_apply_order<4>(n, g, h, xt, w);
        case 5: return guess_apply_order<5>(n, g, h, xt, w);
        case 6: return guess_apply_order<6>(n, g, h, xt, w);
        default: return guess_apply_order<0>(n, g, h, xt, w);
    }
}

__global__ void guess_apply_kernel(size_t n, const double* __restrict__ g, GuessHistory h,
                                   const SolveCtl* __restrict__ sc, double* __restrict__ xt, double* __restrict__ w) {
    guess_apply_body(n, g, h, sc, xt, w);
}

struct GuessCoefTable {
    double c[7][6];
};

// the same with the history's pointers read from the step's table
__global__ void guess_apply_dev_kernel(size_t n, const double* __restrict__ g, const DevHist* __restrict__ dh,
                                       GuessCoefTable cf, const SolveCtl* __restrict__ sc, double* __restrict__ xt,
                                       double* __restrict__ w) {
    GuessHistory h;
    const int avail = dh->avail;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        h.x[j] = j < avail ? dh->x[j] : nullptr;
        h.y[j] = j < avail ? dh->y[j] : nullptr;
    }
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
        for (int j = 0; j < 6; ++j) h.c[q][j] = cf.c[q][j];
    guess_apply_body(n, g, h, sc, xt, w);
}

// The least-squares start (krylov_guess_ls; see guess_gram_body): from the sums in ls[0..31],
// gamma with G gamma = -b, solved on the unit-diagonal scaling of G (a difference whose norm is
// zero is left out) with 1e-6 added to that diagonal -- the sums carry FP32 rounding, and only
// directions closer than that to dependent are damped -- by Cholesky in FP64; the candidate's
// squared residual ||e||^2 + 2 gamma.b + gamma.G gamma; and the coefficients on the stored
// solutions, x0 = sum_j alpha_j x_{n-1-j}, alpha_j = [j = 0] - sum_{p >= max(j,1)} gamma_p (-1)^j C(p, j).
// Writes ls[32] = ||g||^2 (with avail > 0; the plain norm of g is already there otherwise),
// ls[33] = the candidate's squared residual, ls[34..39] = alpha.
__device__ __forceinline__ void ls_solve_body(double* ls, int avail) {
    if (avail <= 0) return;
    const double* sg = ls;
    const int D = avail - 1;
    double gam[5] = {0, 0, 0, 0, 0};
    double r2 = sg[1];
    if (D > 0) {
        double G[5][5], L[5][5], b[5], sc[5];
        bool use[5];
        for (int i = 0; i < D; ++i) {
            b[i] = sg[2 + i];
            for (int j = i; j < D; ++j) G[i][j] = G[j][i] = sg[7 + 5 * i + j];
        }
        for (int i = 0; i < D; ++i) {
            use[i] = isfinite(G[i][i]) && G[i][i] > 0.0;
            sc[i] = use[i] ? 1.0 / sqrt(G[i][i]) : 0.0;
        }
        bool ok = true;
        for (int i = 0; i < D && ok; ++i) {   // Cholesky of the scaled G + 1e-6 I (dropped rows: identity)
            for (int j = 0; j <= i; ++j) {
                double v = (use[i] && use[j]) ? G[i][j] * sc[i] * sc[j] : (i == j ? 1.0 : 0.0);
                if (i == j && use[i]) v += 1e-6;
                for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(v > 0.0)) ok = false;
                    else L[i][i] = sqrt(v);
                } else {
                    L[i][j] = v / L[j][j];
                }
            }
        }
        if (ok) {
            double z[5], t[5];
            for (int i = 0; i < D; ++i) {   // L z = -(scaled b)
                double v = use[i] ? -b[i] * sc[i] : 0.0;
                for (int k = 0; k < i; ++k) v -= L[i][k] * z[k];
                z[i] = v / L[i][i];
            }
            for (int i = D - 1; i >= 0; --i) {   // L^T t = z
                double v = z[i];
                for (int k = i + 1; k < D; ++k) v -= L[k][i] * t[k];
                t[i] = v / L[i][i];
            }
            for (int i = 0; i < D; ++i) gam[i] = use[i] ? t[i] * sc[i] : 0.0;
            double gb = 0.0, ggg = 0.0;
            for (int i = 0; i < D; ++i) {
                gb += gam[i] * b[i];
                double gi = 0.0;
                for (int j = 0; j < D; ++j) gi += G[i][j] * gam[j];
                ggg += gam[i] * gi;
            }
            r2 = sg[1] + 2.0 * gb + ggg;
            if (r2 < 0.0) r2 = 0.0;
        } else {
            for (int i = 0; i < D; ++i) gam[i] = 0.0;
        }
    }
    double* alpha = ls + 34;
    const double binom[6][6] = {{1, 0, 0, 0, 0, 0},  {1, 1, 0, 0, 0, 0},  {1, 2, 1, 0, 0, 0},
                                {1, 3, 3, 1, 0, 0},  {1, 4, 6, 4, 1, 0},  {1, 5, 10, 10, 5, 1}};
    for (int j = 0; j < 6; ++j) {
        double a = j == 0 ? 1.0 : 0.0;
        for (int p = j > 1 ? j : 1; p <= D; ++p) a -= gam[p - 1] * ((j & 1) ? -binom[p][j] : binom[p][j]);
        alpha[j] = j <= D ? a : 0.0;
    }
    ls[32] = sg[0];
    ls[33] = isfinite(r2) ? r2 : INFINITY;
}

__global__ void ls_solve_kernel(double* ls, int avail) { ls_solve_body(ls, avail); }

__global__ void ls_solve_dev_kernel(double* ls, const DevHist* __restrict__ dh) { ls_solve_body(ls, dh->avail); }

// the least-squares start's choice: solve_begin over ls[32] (zero start) and ls[33] (the projection)
__global__ void solve_begin_ls_dev_kernel(const double* __restrict__ ls, const DevHist* __restrict__ dh,
                                          double rtol, double inner_rel, int maxit, GmresCtl* ctl, SolveCtl* sc,
                                          StepStats* ss, double* nrm2) {
    solve_begin_body(ls + 32, dh->avail > 0 ? 1 : 0, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
}

// x~ = x_0 + sum_j (alpha_j - [j = 0]) x_j and w = g - sum_j alpha_j y_j over the Q stored solutions
template <int Q>
__device__ __forceinline__ void apply_alpha(size_t n, const double* __restrict__ g, const DevHist& h,
                                            const double* __restrict__ alpha, double* __restrict__ xt,
                                            double* __restrict__ w) {
    double a[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) a[j] = alpha[j];
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        double xv[Q], yv[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            xv[j] = h.x[j][idx];
            yv[j] = h.y[j][idx];
        }
        double ax = xv[0];
#pragma unroll
        for (int j = 0; j < Q; ++j) ax += (a[j] - (j == 0 ? 1.0 : 0.0)) * xv[j];
        double aw = g[idx];
#pragma unroll
        for (int j = 0; j < Q; ++j) aw += (-a[j]) * yv[j];
        xt[idx] = ax;
        w[idx] = aw;
    }
}

__global__ void guess_apply_ls_dev_kernel(size_t n, const double* __restrict__ g, const DevHist* __restrict__ dh,
                                          const double* __restrict__ ls, const SolveCtl* __restrict__ sc,
                                          double* __restrict__ xt, double* __restrict__ w) {
    const int q = sc->active && sc->guess == 1 ? dh->avail : 0;
    DevHist h = *dh;
    const double* alpha = ls + 34;
    switch (q) {
        case 1: return apply_alpha<1>(n, g, h, alpha, xt, w);
        case 2: return apply_alpha<2>(n, g, h, alpha, xt, w);
        case 3: return apply_alpha<3>(n, g, h, alpha, xt, w);
        case 4: return apply_alpha<4>(n, g, h, alpha, xt, w);
        case 5: return apply_alpha<5>(n, g, h, alpha, xt, w);
        case 6: return apply_alpha<6>(n, g, h, alpha, xt, w);
        default:
            for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
                 idx += (size_t)gridDim.x * blockDim.x) {
                xt[idx] = 0.0;
                w[idx] = g[idx];
            }
    }
}

// The solve's x~ and S~ x~ = g - w into the slot that becomes the newest.
__global__ void hist_store_dev_kernel(size_t n, const double* __restrict__ xt, const double* __restrict__ g,
                                      const double* __restrict__ w, const DevHist* __restrict__ dh) {
    double* __restrict__ xw = dh->xw;
    double* __restrict__ yw = dh->yw;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        xw[idx] = xt[idx];
        yw[idx] = g[idx] - w[idx];
    }
}

// The start of the restart loop: the start residual's squared norm is *nrm_exact when the
// mixed form recomputed it exactly for an extrapolated start, else *nrm2 (the candidate's);
// the loop runs while the residual is above the tolerance.
__global__ void loop_begin_kernel(double* nrm2, const double* __restrict__ nrm_exact, int use_exact,
                                  SolveCtl* sc, StepStats* ss, cudaGraphConditionalHandle loop) {
    if (sc->active && use_exact && sc->guess > 0) *nrm2 = *nrm_exact;
    const double rn = sqrt(*nrm2);
    sc->rnorm = rn;
    unsigned go = sc->active && rn > sc->tol ? 1u : 0u;
    if (sc->active && !isfinite(rn)) {
        ss->nonfinite = 1u;
        go = 0u;
    }
    cudaGraphSetConditional(loop, go);
}

// End of a restart cycle: the host driver's tests on the cycle's true residual, in its order.
__global__ void cycle_end_kernel(const double* __restrict__ nrm2, const GmresCtl* __restrict__ ctl, SolveCtl* sc,
                                 StepStats* ss, double stagnation, cudaGraphConditionalHandle loop) {
    ss->cycles += 1;
    unsigned go = 1u;
    const double rn = sqrt(*nrm2);
    const double prev = sc->rnorm;
    sc->rnorm = rn;
    if (ctl->status != 0 || !isfinite(rn)) {
        ss->nonfinite = 1u;
        go = 0u;
    } else if (rn <= sc->tol) {
        go = 0u;
    } else if (rn <= stagnation * sc->bnorm && rn > 0.5 * prev) {
        go = 0u;
    } else if (ctl->total >= ctl->maxit) {
        ss->notconv = 1u;
        ss->notconv_its = ctl->total;
        ss->notconv_rel = rn / sc->bnorm;
        go = 0u;
    }
    cudaGraphSetConditional(loop, go);
}

// Counters of the finished solve.
__global__ void solve_end_kernel(const GmresCtl* __restrict__ ctl, const SolveCtl* __restrict__ sc, StepStats* ss) {
    const int its = sc->active ? ctl->total : 0;
    ss->its += its;
    ss->last_its = its;
    ss->last_rel = sc->active && sc->bnorm > 0.0 ? sc->rnorm / sc->bnorm : 0.0;
}

int grid_of(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b > 0 ? (int)b : 1;
}

}  // namespace

cudaError_t launch_solve_begin(const double* cand, int avail, double rtol, double inner_rel, int maxit, GmresCtl* ctl,
                               SolveCtl* sc, StepStats* ss, double* nrm2, cudaStream_t s) {
    solve_begin_kernel<<<1, 1, 0, s>>>(cand, avail, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_apply(size_t n, const double* g, const GuessHistory& h, const SolveCtl* sc, double* xt,
                               double* w, cudaStream_t s) {
    guess_apply_kernel<<<grid_of(n), 256, 0, s>>>(n, g, h, sc, xt, w);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_solve_begin_dev(const double* cand, const DevHist* dh, double rtol, double inner_rel, int maxit,
                                   GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double* nrm2, cudaStream_t s) {
    solve_begin_dev_kernel<<<1, 1, 0, s>>>(cand, dh, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_guess_apply_dev(size_t n, const double* g, const DevHist* dh, const double (*coef)[6],
                                   const SolveCtl* sc, double* xt, double* w, cudaStream_t s) {
    GuessCoefTable cf;
    for (int q = 0; q < 7; ++q)
        for (int j = 0; j < 6; ++j) cf.c[q][j] = coef[q][j];
    guess_apply_dev_kernel<<<grid_of(n), 256, 0, s>>>(n, g, dh, cf, sc, xt, w);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ls_solve(double* ls, int avail, cudaStream_t s) {
    ls_solve_kernel<<<1, 1, 0, s>>>(ls, avail);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ls_start_dev(size_t n, const double* g, const DevHist* dh, double* ls, double rtol,
                                double inner_rel, int maxit, GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double* nrm2,
                                double* xt, double* w, cudaStream_t s) {
    ls_solve_dev_kernel<<<1, 1, 0, s>>>(ls, dh);
    solve_begin_ls_dev_kernel<<<1, 1, 0, s>>>(ls, dh, rtol, inner_rel, maxit, ctl, sc, ss, nrm2);
    guess_apply_ls_dev_kernel<<<grid_of(n), 256, 0, s>>>(n, g, dh, ls, sc, xt, w);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_hist_store_dev(size_t n, const double* xt, const double* g, const double* w, const DevHist* dh,
                                  cudaStream_t s) {
    hist_store_dev_kernel<<<grid_of(n), 256, 0, s>>>(n, xt, g, w, dh);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_loop_begin(double* nrm2, const double* nrm_exact, int use_exact, SolveCtl* sc, StepStats* ss,
                              cudaGraphConditionalHandle loop, cudaStream_t s) {
    loop_begin_kernel<<<1, 1, 0, s>>>(nrm2, nrm_exact, use_exact, sc, ss, loop);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cycle_end(const double* nrm2, const GmresCtl* ctl, SolveCtl* sc, StepStats* ss, double stagnation,
                             cudaGraphConditionalHandle loop, cudaStream_t s) {
    cycle_end_kernel<<<1, 1, 0, s>>>(nrm2, ctl, sc, ss, stagnation, loop);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_solve_end(const GmresCtl* ctl, const SolveCtl* sc, StepStats* ss, cudaStream_t s) {
    solve_end_kernel<<<1, 1, 0, s>>>(ctl, sc, ss);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hdgdg
