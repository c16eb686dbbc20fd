// HDG implicit-stage operators: setup (local inverses, condensed trace matrix) and the
// per-stage condensation and recovery kernels.
//
// Stage system (Sec. 6, eq. linearizedHDGsystem): [[A, B], [C, D]] [Q; Qhat] = [R1; 0] with
//   A = I - dt a M^{-1} dL/dQ,  B = -dt a M^{-1} dL/dQhat,  C = dFlx/dQ,  D = dFlx/dQhat,
// L(q, qhat) = (F_L, grad v) + (s, v) - <Fhat_L . n, v> (eq. SemiDiscretizedForm_ode) and
// the hybridised Lax-Friedrichs flux of eq. linear_hdgflux3,
//   n . Fhat_L = (n.U + tau (phi - phi_hat), n_x phi_B phi + tau (U - U_hat),
//                 n_y phi_B phi + tau (V - V_hat)),  tau = max_pm sqrt(phi_B).
// With collocated GLL faces the conservation condition (eq. HDGcont) holds node by node;
// this library keeps its rows in pointwise form (divided by the face weight (h/2) w_b), so
//   C rows at a face node of an element: (n_x U + n_y V + tau phi, n_x phi_B phi + tau U,
//   n_y phi_B phi + tau V), and D = -tau per side (diagonal).
// B acts only on boundary volume nodes: B = -beta tau with beta = dt a (2/h) / w_0.
// Schur complement (eq. linearizedHDGsystem_schur): S = D - C A^{-1} B, rhs -C A^{-1} R1;
// recovery (eq. recover_volume_unknowns): Q = A^{-1}(R1 - B Qhat).
#include <type_traits>

#include "compensated.h"
#include "internal.h"
#include "schur.h"
#include "staged.h"
#include "ens.h"

namespace hdgdg {
namespace {

// In-place Gauss-Jordan inversion of the n x n matrix in the left half of the row-major
// augmented array M[n][2n] (right half must hold I); partial pivoting; whole CTA.
// On return the right half holds the inverse.  *singular set if a pivot is 0.
__device__ void gauss_jordan(double* M, int n, int* singular, int* s_piv) {
    const int ld = 2 * n;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            double best = fabs(M[k * ld + k]);
            for (int r = k + 1; r < n; ++r) {
                const double v = fabs(M[r * ld + k]);
                if (v > best) { best = v; p = r; }
            }
            *s_piv = p;
            if (best == 0.0) *singular = 1;
        }
        __syncthreads();
        const int p = *s_piv;
        if (p != k) {
            for (int c = threadIdx.x; c < ld; c += blockDim.x) {
                const double t = M[k * ld + c];
                M[k * ld + c] = M[p * ld + c];
                M[p * ld + c] = t;
            }
            __syncthreads();
        }
        const double piv = M[k * ld + k];
        __syncthreads();
        const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
        for (int c = threadIdx.x; c < ld; c += blockDim.x) M[k * ld + c] *= inv;
        __syncthreads();
        for (int t = threadIdx.x; t < n * ld; t += blockDim.x) {
            const int r = t / ld, c = t % ld;
            if (r == k || c == k) continue;
            M[r * ld + c] -= M[r * ld + k] * M[k * ld + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != k) M[r * ld + k] = 0.0;
        __syncthreads();
    }
}

// One CTA per element.  Builds A_e, inverts it, writes A^{-1} (column major) and the
// element Schur block S_e = D_e - C_e A^{-1} B_e in local trace order (f, c, b).
// The augmented matrix lives in shared memory when it fits (k <= 5); above that it lives in
// a global workspace of one [NV][2 NV] slab per CTA (gwork, elements e0 .. e0 + gridDim.x).
template <int P, bool GMEM>
__global__ void build_local_kernel(Geom g, const double* __restrict__ phiB,
                                   const double* __restrict__ tau_edge, double dta,
                                   double* __restrict__ Ainv, double* __restrict__ Se,
                                   int* singular, int e0, double* __restrict__ gwork) {
    constexpr int Np = P * P, NV = 3 * Np, NT = 12 * P;
    extern __shared__ double sm[];
    double* M = GMEM ? gwork + (size_t)blockIdx.x * NV * 2 * NV : sm;   // [NV][2 NV]
    double* pb = GMEM ? sm : M + NV * 2 * NV;                              // [Np]
    double* tau = pb + Np;                                                 // [4][P]
    __shared__ int s_piv;
    const int e = e0 + blockIdx.x;
    const int ld = 2 * NV;
    dta *= dt_factor(g, e);   // this instance's time step

    for (int n = threadIdx.x; n < Np; n += blockDim.x) pb[n] = phiB[(size_t)e * Np + n];
    for (int t = threadIdx.x; t < 4 * P; t += blockDim.x)
        tau[t] = tau_edge[(size_t)edge_of_face(e, t / P, g) * P + t % P];
    for (int t = threadIdx.x; t < NV * ld; t += blockDim.x) {
        const int r = t / ld, c = t % ld;
        M[t] = (c == r || c == r + NV) ? 1.0 : 0.0;
    }
    __syncthreads();

    // A = I - dta * d(M^{-1} L)/dQ, one row per thread
    const double th = g.two_over_h;
    for (int r = threadIdx.x; r < NV; r += blockDim.x) {
        const int c = r / Np, n = r % Np, i = n % P, j = n / P;
        double* row = M + r * ld;
        if (c == 0) {   // phi row: volume term of (U, V) fluxes
            for (int a = 0; a < P; ++a) {
                row[1 * Np + j * P + a] -= dta * th * g.Dhat[i * P + a];
                row[2 * Np + a * P + i] -= dta * th * g.Dhat[j * P + a];
            }
        } else if (c == 1) {   // U row: volume term of phi_eta phi_B along x, source phi_eta d_x phi_B
            double dB = 0.0;
            for (int a = 0; a < P; ++a) {
                row[0 * Np + j * P + a] -= dta * th * g.Dhat[i * P + a] * pb[j * P + a];
                dB += g.D[i * P + a] * pb[j * P + a];
            }
            row[0 * Np + n] -= dta * th * dB;
        } else {   // V row
            double dB = 0.0;
            for (int a = 0; a < P; ++a) {
                row[0 * Np + a * P + i] -= dta * th * g.Dhat[j * P + a] * pb[a * P + i];
                dB += g.D[j * P + a] * pb[a * P + i];
            }
            row[0 * Np + n] -= dta * th * dB;
        }
        // faces through the node: -(2/h)/w0 * d(Fhat.n)/dQ, with the minus sign of -<.,.>
        const double lift = th * g.inv_w0;
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const double t = tau[f * P + b];
            const double nx = f == 0 ? -1.0 : f == 1 ? 1.0 : 0.0;
            const double ny = f == 2 ? -1.0 : f == 3 ? 1.0 : 0.0;
            // M^{-1} L contains -lift * (Fhat . n); A = I - dta M^{-1} dL/dQ adds +dta*lift*d(Fhat.n)/dQ
            const double k = dta * lift;
            if (c == 0) {
                row[1 * Np + n] += k * nx;
                row[2 * Np + n] += k * ny;
                row[0 * Np + n] += k * t;
            } else if (c == 1) {
                row[0 * Np + n] += k * nx * pb[n];
                row[1 * Np + n] += k * t;
            } else {
                row[0 * Np + n] += k * ny * pb[n];
                row[2 * Np + n] += k * t;
            }
        }
    }
    __syncthreads();
    gauss_jordan(M, NV, singular, &s_piv);

    // A^{-1}[r][s] = M[r][NV + s]; store column major
    double* Ae = Ainv + (size_t)e * NV * NV;
    for (int t = threadIdx.x; t < NV * NV; t += blockDim.x) {
        const int s = t / NV, r = t % NV;
        Ae[t] = M[r * ld + NV + s];
    }

    // S_e[(f1,c1,b1)][(f2,c2,b2)] = -tau1 delta + beta tau2 (C-row combination of A^{-1})
    const double beta = dta * th * g.inv_w0;
    double* S = Se + (size_t)e * NT * NT;
    for (int t = threadIdx.x; t < NT * NT; t += blockDim.x) {
        const int rr = t / NT, cc = t % NT;
        const int f1 = rr / (3 * P), c1 = (rr / P) % 3, b1 = rr % P;
        const int f2 = cc / (3 * P), c2 = (cc / P) % 3, b2 = cc % P;
        const int n1 = face_node(f1, b1, P), n2 = face_node(f2, b2, P);
        const double t1 = tau[f1 * P + b1], t2 = tau[f2 * P + b2];
        const double nx = f1 == 0 ? -1.0 : f1 == 1 ? 1.0 : 0.0;
        const double ny = f1 == 2 ? -1.0 : f1 == 3 ? 1.0 : 0.0;
        const int col = NV + c2 * Np + n2;
        const double aph = M[(0 * Np + n1) * ld + col];
        const double aU = M[(1 * Np + n1) * ld + col];
        const double aV = M[(2 * Np + n1) * ld + col];
        double cz, d = t1;
        if (neighbour(e, f1, g) >= 0 || g.dirichlet) {   // (Dirichlet rows are replaced at assembly)
            if (c1 == 0) cz = nx * aU + ny * aV + t1 * aph;
            else if (c1 == 1) cz = nx * pb[n1] * aph + t1 * aU;
            else cz = ny * pb[n1] * aph + t1 * aV;
        } else {
            // wall face: the element's share plus its mirror's (state R q, normal -n), i.e.
            // 2 (n.U + tau phi) for phi_hat, 2 tau U_tangential for the momentum rows, D = -2 tau
            const double un = nx * aU + ny * aV;
            if (c1 == 0) cz = 2.0 * (un + t1 * aph);
            else if (c1 == 1) cz = 2.0 * t1 * (aU - un * nx);
            else cz = 2.0 * t1 * (aV - un * ny);
            d = 2.0 * t1;
        }
        double v = beta * t2 * cz;
        if (rr == cc) v -= d;
        S[t] = v;
    }
}

// One CTA per edge: gathers the 7 blocks of its row of S from the two elements' S_e.
// S7 layout [edge][slot][row ii][col jj] (row major), slot 0 = diagonal block.
template <int P>
__global__ void gather_rows_kernel(Geom g, const double* __restrict__ Se, double* __restrict__ S7,
                                   double* __restrict__ Srr, int* __restrict__ Scol) {
    constexpr int NF = 3 * P, NT = 12 * P;
    const int r = blockIdx.x;
    int em, fm, ep, fp;
    edge_sides(r, g, &em, &fm, &ep, &fp);
    // a wall edge has one element: its slots carry that element's blocks, the absent side's
    // three slots are zero blocks pointing at the edge itself
    const double* Sm = em >= 0 ? Se + (size_t)em * NT * NT : nullptr;
    const double* Sp = ep >= 0 ? Se + (size_t)ep * NT * NT : nullptr;
    double* row = S7 + (size_t)r * 7 * NF * NF;
    for (int t = threadIdx.x; t < 7 * NF * NF; t += blockDim.x) {
        const int slot = t / (NF * NF), ii = (t / NF) % NF, jj = t % NF;
        double v = 0.0;
        if (g.dirichlet && (!Sm || !Sp)) {
            v = (slot == 0 && ii == jj) ? 1.0 : 0.0;   // prescribed trace: qhat = q_bc
        } else if (slot == 0) {
            if (Sm) v += Sm[(fm * NF + ii) * NT + fm * NF + jj];
            if (Sp) v += Sp[(fp * NF + ii) * NT + fp * NF + jj];
        } else {
            const int side = (slot - 1) / 3, k = (slot - 1) % 3;
            const int fs = side == 0 ? fm : fp;
            const int fo = k < fs ? k : k + 1;        // k-th face other than fs, ascending
            const double* Sx = side == 0 ? Sm : Sp;
            if (Sx) v = Sx[(fs * NF + ii) * NT + fo * NF + jj];
        }
        row[t] = v;
        if (slot == 0) Srr[(size_t)r * NF * NF + jj * NF + ii] = v;   // column major copy
    }
    if (threadIdx.x < 6) {
        const int slot = threadIdx.x + 1;
        const int side = (slot - 1) / 3, k = (slot - 1) % 3;
        const int fs = side == 0 ? fm : fp;
        const int fo = k < fs ? k : k + 1;
        const int el = side == 0 ? em : ep;
        const bool prescribed = g.dirichlet && (em < 0 || ep < 0);
        Scol[(size_t)r * 6 + threadIdx.x] = (el >= 0 && !prescribed) ? edge_of_face(el, fo, g) : r;
    }
}

// One CTA per edge: M^{-1} = S_rr^{-1}, stored column major.
template <int P>
__global__ void invert_diag_kernel(const double* __restrict__ S7, double* __restrict__ Minv,
                                   int* singular) {
    constexpr int NF = 3 * P;
    __shared__ double M[NF * 2 * NF];
    __shared__ int s_piv;
    const int r = blockIdx.x;
    const double* blk = S7 + (size_t)r * 7 * NF * NF;
    for (int t = threadIdx.x; t < NF * 2 * NF; t += blockDim.x) {
        const int ii = t / (2 * NF), c = t % (2 * NF);
        M[t] = c < NF ? blk[ii * NF + c] : (c - NF == ii ? 1.0 : 0.0);
    }
    __syncthreads();
    gauss_jordan(M, NF, singular, &s_piv);
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) {
        const int jj = t / NF, ii = t % NF;
        Minv[(size_t)r * NF * NF + t] = M[ii * 2 * NF + NF + jj];
    }
}

// S~[r][slot] = S[r][slot] M^{-1}_{col}, slots 1..6, stored [edge][slot-1][col jj][row ii].
template <int P>
__global__ void precondition_kernel(int n_edges, const double* __restrict__ S7,
                                    const double* __restrict__ Minv, const int* __restrict__ Scol,
                                    double* __restrict__ Stil) {
    constexpr int NF = 3 * P;
    const int r = blockIdx.x;
    for (int t = threadIdx.x; t < 6 * NF * NF; t += blockDim.x) {
        const int sl = t / (NF * NF), jj = (t / NF) % NF, ii = t % NF;
        const double* S = S7 + ((size_t)r * 7 + sl + 1) * NF * NF;           // row major
        const double* Mi = Minv + (size_t)Scol[(size_t)r * 6 + sl] * NF * NF;  // column major
        double acc = 0.0;
        for (int k = 0; k < NF; ++k) acc += S[ii * NF + k] * Mi[jj * NF + k];
        Stil[((size_t)r * 6 + sl) * NF * NF + jj * NF + ii] = acc;
    }
}

// Z = A^{-1} R1: one thread per (element, row); R1 staged in shared memory.  T is the type of
// the stored operator and of the products and sums (double, or float for the FP32 variant).
template <int P, typename T>
__global__ void apply_ainv_kernel(Geom g, const T* __restrict__ Ainv, const double* __restrict__ R1,
                                  double* __restrict__ Z) {
    constexpr int Np = P * P, NV = 3 * Np;
    constexpr int EPB = (256 / NV) > 0 ? 256 / NV : 1;
    __shared__ T sx[EPB][NV];
    const int le = threadIdx.x / NV, r = threadIdx.x % NV;
    const int e = blockIdx.x * EPB + le;
    const size_t fs = (size_t)g.n_el * Np;
    const bool live = e < g.n_el && le < EPB;
    if (live) sx[le][r] = (T)R1[(r / Np) * fs + (size_t)e * Np + r % Np];
    __syncthreads();
    if (!live) return;
    const T* A = Ainv + (size_t)e * NV * NV;
    T acc = 0;
#pragma unroll 8
    for (int s = 0; s < NV; ++s) acc += A[s * NV + r] * sx[le][s];
    Z[(r / Np) * fs + (size_t)e * Np + r % Np] = (double)acc;
}

// ---- FP64-class local contractions on the FP32 pipes (compensated.h) ---------------------------
__global__ void split_kernel(const double* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo,
                             size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        split(a[i], hi[i], lo[i]);
}

// Z = A^{-1} R1 with the FP32-pair operator: one thread per (element, row), as apply_ainv_kernel;
// EPB elements per block (the tile the autotuner picks; results do not depend on it).
template <int P, int EPB>
__global__ void apply_ainv_x2_kernel(Geom g, const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                     const double* __restrict__ R1, double* __restrict__ Z) {
    constexpr int Np = P * P, NV = 3 * Np;
    __shared__ float sxh[EPB][NV], sxl[EPB][NV];
    const int le = threadIdx.x / NV, r = threadIdx.x % NV;
    const int e = blockIdx.x * EPB + le;
    const size_t fs = (size_t)g.n_el * Np;
    const bool live = e < g.n_el && le < EPB;
    if (live) split(R1[(r / Np) * fs + (size_t)e * Np + r % Np], sxh[le][r], sxl[le][r]);
    __syncthreads();
    if (!live) return;
    const size_t base = (size_t)e * NV * NV;
    Dot2 acc;
#pragma unroll 4
    for (int s = 0; s < NV; ++s) acc.add(Ahi[base + s * NV + r], Alo[base + s * NV + r], sxh[le][s], sxl[le][s]);
    Z[(r / Np) * fs + (size_t)e * Np + r % Np] = acc.value();
}

// Q = Z + beta A^{-1}_{:, boundary} (tau qhat), Lst = (Q - R1) / a_ii with the FP32-pair operator;
// EPB elements per block as above.
template <int P, int EPB>
__global__ void recover_x2_kernel(Geom g, const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                  const double* __restrict__ Z, const double* __restrict__ R1,
                                  const double* __restrict__ tau_edge, const double* __restrict__ qhat, double beta,
                                  double inv_aii, double* __restrict__ Q, double* __restrict__ Lst) {
    constexpr int Np = P * P, NV = 3 * Np, NF = 3 * P;
    __shared__ float suh[EPB][NV], sul[EPB][NV];
    const int le = threadIdx.x / NV, r = threadIdx.x % NV;
    const int e = blockIdx.x * EPB + le;
    const size_t fs = (size_t)g.n_el * Np;
    const bool live = e < g.n_el && le < EPB;
    if (live) {
        const int c = r / Np, n = r % Np, i = n % P, j = n / P;
        double u = 0.0;
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const int ed = edge_of_face(e, f, g);
            u += tau_edge[(size_t)ed * P + b] * qhat[(size_t)ed * NF + c * P + b];
        }
        split(u, suh[le][r], sul[le][r]);
    }
    __syncthreads();
    if (!live) return;
    const size_t base = (size_t)e * NV * NV;
    Dot2 acc;
    for (int c = 0; c < 3; ++c) {
        for (int n = 0; n < Np; ++n) {
            const int i = n % P, j = n / P;
            if (i != 0 && i != P - 1 && j != 0 && j != P - 1) continue;
            const int s = c * Np + n;
            acc.add(Ahi[base + s * NV + r], Alo[base + s * NV + r], suh[le][s], sul[le][s]);
        }
    }
    const size_t o = (r / Np) * fs + (size_t)e * Np + r % Np;
    const double q = Z[o] + beta * dt_factor(g, e) * acc.value();
    Q[o] = q;
    Lst[o] = (q - R1[o]) * inv_aii;
}

// g = -C Z at every trace node: one thread per (edge, b).
template <int P>
__device__ __forceinline__ void edge_rhs_body(int bid, const Geom& g, const double* __restrict__ Z,
                                              const double* __restrict__ phiB, const double* __restrict__ tau_edge,
                                              double* __restrict__ gvec, double t_bc) {
    constexpr int Np = P * P, NF = 3 * P;
    const int t = bid * 256 + threadIdx.x;
    if (t >= g.n_edges * P) return;
    const int r = t / P, b = t % P;
    int em, fm, ep, fp;
    edge_sides(r, g, &em, &fm, &ep, &fp);
    const size_t fs = (size_t)g.n_el * Np;
    const double tau = tau_edge[(size_t)r * P + b];
    const bool xedge = fm == 1;
    double* out = gvec + (size_t)r * NF;
    const int e_in = em >= 0 ? em : ep, f_in = em >= 0 ? fm : fp;   // an element that exists
    if (g.dirichlet && (em < 0 || ep < 0)) {   // prescribed trace row: qhat = q_bc(t)
        double x, y, ph, U, V;
        face_node_xy(g, e_in, f_in, b, &x, &y);
        vortex_state(g, x, y, t_bc * dt_factor(g, e_in), &ph, &U, &V);
        out[b] = ph;
        out[P + b] = U;
        out[2 * P + b] = V;
        return;
    }
    // face values of the two sides, the momentum as normal (n) and tangential (t) components along
    // the edge's +axis; a wall's absent side is the mirror of the other (same phi and tangential
    // momentum, opposite normal momentum)
    double zph[2], zn[2], zt[2], pb[2];
    for (int side = 0; side < 2; ++side) {
        int e = side == 0 ? em : ep;
        const int f = side == 0 ? fm : fp;
        const bool mirror = e < 0;
        if (mirror) e = e_in;
        const size_t o = (size_t)e * Np + face_node(mirror ? f_in : f, b, P);
        const double zU = Z[fs + o], zV = Z[2 * fs + o];
        zph[side] = Z[o];
        pb[side] = phiB[o];
        zn[side] = mirror ? -(xedge ? zU : zV) : (xedge ? zU : zV);
        zt[side] = xedge ? zV : zU;
    }
    // g = -(C_- Z_- + C_+ Z_+), the normal +1 on the minus side and -1 on the plus side:
    //   phi_hat row: -(n.U + tau phi) summed;  normal row: -(n phi_B phi + tau U_n);  tangential: -tau U_t
    const double g0 = (zn[1] - zn[0]) - tau * (zph[0] + zph[1]);
    const double gn = (pb[1] * zph[1] - pb[0] * zph[0]) - tau * (zn[0] + zn[1]);
    const double gt = -tau * (zt[0] + zt[1]);
    out[b] = g0;
    out[(xedge ? 1 : 2) * P + b] = gn;
    out[(xedge ? 2 : 1) * P + b] = gt;
}

template <int P>
__global__ void __launch_bounds__(256)
edge_rhs_kernel(Geom g, const double* __restrict__ Z, const double* __restrict__ phiB,
                const double* __restrict__ tau_edge, double* __restrict__ gvec, double t_bc) {
    edge_rhs_body<P>(blockIdx.x, g, Z, phiB, tau_edge, gvec, t_bc);
}

// Q = Z + beta A^{-1}_{:, boundary} (tau qhat);  Lst = (Q - R1) * inv_aii.  T as above.
template <int P, typename T>
__global__ void recover_kernel(Geom g, const T* __restrict__ Ainv, const double* __restrict__ Z,
                               const double* __restrict__ R1, const double* __restrict__ tau_edge,
                               const double* __restrict__ qhat, double beta, double inv_aii,
                               double* __restrict__ Q, double* __restrict__ Lst) {
    constexpr int Np = P * P, NV = 3 * Np, NF = 3 * P;
    constexpr int EPB = (256 / NV) > 0 ? 256 / NV : 1;
    __shared__ T su[EPB][NV];
    const int le = threadIdx.x / NV, r = threadIdx.x % NV;
    const int e = blockIdx.x * EPB + le;
    const size_t fs = (size_t)g.n_el * Np;
    const bool live = e < g.n_el && le < EPB;
    if (live) {
        const int c = r / Np, n = r % Np, i = n % P, j = n / P;
        double u = 0.0;
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const int ed = edge_of_face(e, f, g);
            u += tau_edge[(size_t)ed * P + b] * qhat[(size_t)ed * NF + c * P + b];
        }
        su[le][r] = (T)u;
    }
    __syncthreads();
    if (!live) return;
    const T* A = Ainv + (size_t)e * NV * NV;
    T acc = 0;
    for (int c = 0; c < 3; ++c) {
        for (int n = 0; n < Np; ++n) {
            const int i = n % P, j = n / P;
            if (i != 0 && i != P - 1 && j != 0 && j != P - 1) continue;
            const int s = c * Np + n;
            acc += A[s * NV + r] * su[le][s];
        }
    }
    const size_t o = (r / Np) * fs + (size_t)e * Np + r % Np;
    const double q = Z[o] + beta * dt_factor(g, e) * (double)acc;
    Q[o] = q;
    Lst[o] = (q - R1[o]) * inv_aii;
}

// ---- Local solves through the Schur complement on phi ---------------------------------------------
// With collocated GLL nodes the velocity blocks of A are diagonal and equal to the phi block's
// diagonal d_n = 1 + kk sum_{faces at n} tau:
//   A = [[diag(d), Bx, By], [Cx, diag(d), 0], [Cy, 0, diag(d)]],
//   (Bx v)_(i,j) = sum_a E[i][a] v_(a,j),   E = alpha Dhat + kk diag(nv),
//   (Cx v)_(i,j) = sum_a G[i][a] phi_B v_(a,j) + cx_(i,j) v_(i,j),   G = alpha Dhat,
//   cx = alpha (d_x phi_B) + kk nv(i) phi_B,
// alpha = -dta (2/h), kk = dta (2/h) / w_0, nv(i) = [i = P-1] - [i = 0] the outward normal of the
// element's x-face through the node (By, Cy alike along y with the same E and G, cy with nv(j);
// these are the rows build_local_kernel fills).  Eliminating U and V:
//   S phi = x_phi - Bx d^{-1} x_U - By d^{-1} x_V,   S = diag(d) - Bx d^{-1} Cx - By d^{-1} Cy,
//   U = d^{-1} (x_U - Cx phi),   V = d^{-1} (x_V - Cy phi),
// and S^{-1} is the (phi, phi) block of A^{-1}.  Per element the kernels read Np^2 + 4 Np numbers
// of operator data instead of (3 Np)^2; E and G depend only on the instance's time step.  Each
// output is one dot product: s over 2P + 1 terms, phi over Np, d U and d V over P + 2.

// Setup, one thread per (element, node n): row n of the (phi, phi) block of A^{-1} into
// S [n_el][col m][row n], and aux [n_el][4][Np] = (1/d, -cx, -cy, phi_B) at node n.
template <int P, class A>
__global__ void schur_setup_kernel(Geom g, const double* __restrict__ Ainv, const double* __restrict__ phiB,
                                   const double* __restrict__ tau_edge, double dta, typename A::T* __restrict__ S,
                                   typename A::T* __restrict__ aux) {
    constexpr int Np = P * P, NV = 3 * Np;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)g.n_el * Np) return;
    const int e = (int)(t / Np), n = (int)(t % Np), i = n % P, j = n / P;
    const double* Ae = Ainv + (size_t)e * NV * NV;
    for (int m = 0; m < Np; ++m)   // (A^{-1})_{n m}; A^{-1} is stored column major
        store_from<A>(&S[((size_t)e * Np + m) * Np + n], Ae[(size_t)m * NV + n]);
    const double de = dta * dt_factor(g, e), th = g.two_over_h;
    const double alpha = -de * th, kk = de * th * g.inv_w0;
    double tsum = 0.0;
    for (int f = 0; f < 4; ++f) {
        const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                        (f == 3 && j == P - 1);
        if (on) tsum += tau_edge[(size_t)edge_of_face(e, f, g) * P + ((f < 2) ? j : i)];
    }
    const double* pb = phiB + (size_t)e * Np;
    double dBx = 0.0, dBy = 0.0;
    for (int a = 0; a < P; ++a) {
        dBx += g.D[i * P + a] * pb[j * P + a];
        dBy += g.D[j * P + a] * pb[a * P + i];
    }
    const double nx = (i == P - 1 ? 1.0 : 0.0) - (i == 0 ? 1.0 : 0.0);
    const double ny = (j == P - 1 ? 1.0 : 0.0) - (j == 0 ? 1.0 : 0.0);
    typename A::T* ax = aux + (size_t)e * 4 * Np;
    store_from<A>(&ax[n], 1.0 / (1.0 + kk * tsum));
    store_from<A>(&ax[Np + n], -(alpha * dBx + kk * nx * pb[n]));
    store_from<A>(&ax[2 * Np + n], -(alpha * dBy + kk * ny * pb[n]));
    store_from<A>(&ax[3 * Np + n], pb[n]);
}

// Setup, one thread per (instance, entry): EG [batch][2][P][P] = (-E, -G) of each instance.
template <int P, class A>
__global__ void schur_eg_kernel(Geom g, double dta, typename A::T* __restrict__ EG) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.batch * 2 * P * P) return;
    const int inst = t / (2 * P * P), w = (t / (P * P)) % 2, r = (t % (P * P)) / P, a = t % P;
    const double de = dta * dt_factor(g, inst * g.n_el_inst), th = g.two_over_h;
    const double alpha = -de * th, kk = de * th * g.inv_w0;
    double v = alpha * g.Dhat[r * P + a];
    if (w == 0 && a == r) v += kk * ((r == P - 1 ? 1.0 : 0.0) - (r == 0 ? 1.0 : 0.0));
    store_from<A>(&EG[t], -v);
}


// The three fields of R1 at node o (field stride fs): read, or (src.base set) formed term by term
// as launch_combine forms them and written back to R1.  Every load is issued before the first
// store so that they overlap (the terms' pointers sit in a struct: the compiler cannot prove that
// the stores to R1 leave them alone).
__device__ __forceinline__ void r1_fields(const double* __restrict__ R1, const R1Source& src, size_t o, size_t fs,
                                          double v[3]) {
    if (!src.base) {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = R1[o + c * fs];
        return;
    }
    double x[kR1FusedTerms][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = src.base[o + c * fs];
#pragma unroll
    for (int k = 0; k < kR1FusedTerms; ++k)   // constant indices keep the terms in the parameter bank
        if (k < src.t.n) {
#pragma unroll
            for (int c = 0; c < 3; ++c) x[k][c] = src.t.X[k][o + c * fs];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int k = 0; k < kR1FusedTerms; ++k)
            if (k < src.t.n) v[c] += src.t.c[k] * x[k][c];
        const_cast<double*>(R1)[o + c * fs] = v[c];
    }
}

// Z = A^{-1} R1 through the Schur complement: one thread per (element, node), EPB elements per block.
template <int P, int EPB, class A>
__device__ __forceinline__ void schur_condense_body(int bid, const Geom& g, const typename A::T* __restrict__ S,
                                                    const typename A::T* __restrict__ aux,
                                                    const typename A::T* __restrict__ EG,
                                                    const double* __restrict__ R1, double* __restrict__ Z,
                                                    const R1Source& src = R1Source{}) {
    using T = typename A::T;
    constexpr int Np = P * P;
    __shared__ SchurSmem<P, EPB, A> sm;
    const int le = threadIdx.x / Np, n = threadIdx.x % Np;
    const int e = bid * EPB + le;
    const bool live = le < EPB && e < g.n_el;
    const size_t fs = (size_t)g.n_el * Np, o = (size_t)e * Np + n;
    T x0{}, xU{}, xV{};
    if (live) {
        double r[3];
        r1_fields(R1, src, o, fs, r);
        x0 = A::from(r[0]);
        xU = A::from(r[1]);
        xV = A::from(r[2]);
    }
    T phi{}, U{}, V{};
    schur_solve<P, EPB, A>(sm, g, e, le, n, live, S, aux, EG, x0, xU, xV, phi, U, V);
    if (live) {
        Z[o] = A::to(phi);
        Z[fs + o] = A::to(U);
        Z[2 * fs + o] = A::to(V);
    }
}

template <int P, int EPB, class A>
__global__ void __launch_bounds__(EPB * P * P)
    schur_condense_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                          const typename A::T* __restrict__ EG, const double* __restrict__ R1,
                          double* __restrict__ Z, R1Source src) {
    schur_condense_body<P, EPB, A>(blockIdx.x, g, S, aux, EG, R1, Z, src);
}

// Q = Z + beta A^{-1} (tau qhat), Lst = Q - R1 (= dt a_ii M^{-1} L; inv_aii must be 1: the
// callers fold 1/a_ii into the stage combinations) through the Schur complement.
template <int P, int EPB, class A>
__device__ __forceinline__ void schur_recover_body(int bid, const Geom& g, const typename A::T* __restrict__ S,
                                                   const typename A::T* __restrict__ aux,
                                                   const typename A::T* __restrict__ EG, const double* __restrict__ Z,
                                                   const double* __restrict__ R1, const double* __restrict__ tau_edge,
                                                   const double* __restrict__ qhat, double beta, double inv_aii,
                                                   double* __restrict__ Q, double* __restrict__ Lst,
                                                   float* __restrict__ Q32 = nullptr) {
    using T = typename A::T;
    constexpr int Np = P * P, NF = 3 * P;
    __shared__ SchurSmem<P, EPB, A> sm;
    const int le = threadIdx.x / Np, n = threadIdx.x % Np, i = n % P, j = n / P;
    const int e = bid * EPB + le;
    const bool live = le < EPB && e < g.n_el;
    const size_t fs = (size_t)g.n_el * Np, o = (size_t)e * Np + n;
    double u[3] = {0.0, 0.0, 0.0};
    if (live) {
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const int ed = edge_of_face(e, f, g);
            const double tau = tau_edge[(size_t)ed * P + b];
            for (int c = 0; c < 3; ++c) u[c] += tau * qhat[(size_t)ed * NF + c * P + b];
        }
    }
    T y[3];
    schur_solve<P, EPB, A>(sm, g, e, le, n, live, S, aux, EG, A::from(u[0]), A::from(u[1]), A::from(u[2]), y[0],
                           y[1], y[2]);
    if (live) {
        const double kk = beta * dt_factor(g, e);
        for (int c = 0; c < 3; ++c) {
            const size_t oc = c * fs + o;
            const double q = Z[oc] + kk * A::to(y[c]);
            if (Q32) Q32[oc] = f64_to_f32(q);   // the FP32 stage value the mixed form's DG residual reads
            else Q[oc] = q;
            Lst[oc] = q - R1[oc];   // callers fold 1/a_ii into the stage combinations (inv_aii = 1)
        }
    }
}

template <int P, int EPB, class A>
__global__ void __launch_bounds__(EPB * P * P)
    schur_recover_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                         const typename A::T* __restrict__ EG, const double* __restrict__ Z,
                         const double* __restrict__ R1, const double* __restrict__ tau_edge,
                         const double* __restrict__ qhat, double beta, double inv_aii, double* __restrict__ Q,
                         double* __restrict__ Lst, float* __restrict__ Q32) {
    schur_recover_body<P, EPB, A>(blockIdx.x, g, S, aux, EG, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, Q32);
}

// The same two passes with the element operators staged into shared memory by bulk copies
// (staged.h) while each thread loads its own stage data and traces: the arithmetic is the
// kernels' above, operand for operand.  err: the handle's word for a wait that ran out.
template <int P, int EPB, class A>
__global__ void __launch_bounds__(EPB * P * P)
    schur_condense_staged_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                                 const typename A::T* __restrict__ EG, const double* __restrict__ R1,
                                 double* __restrict__ Z, unsigned* err, R1Source src) {
    using T = typename A::T;
    constexpr int Np = P * P;
    __shared__ SchurSmem<P, EPB, A> sm;
    __shared__ StagedOps<P, EPB, A> so;
    const int le = threadIdx.x / Np, n = threadIdx.x % Np;
    const int e0 = blockIdx.x * EPB, e = e0 + le;
    const int ne = g.n_el - e0 < EPB ? g.n_el - e0 : EPB;
    const bool live = le < EPB && e < g.n_el;
    so.issue(S, aux, e0, ne);
    const size_t fs = (size_t)g.n_el * Np, o = (size_t)e * Np + n;
    T x0{}, xU{}, xV{};
    if (live) {
        double r[3];
        r1_fields(R1, src, o, fs, r);
        x0 = A::from(r[0]);
        xU = A::from(r[1]);
        xV = A::from(r[2]);
    }
    if (!so.wait(err)) return;
    SchurNode<A> nd;
    if (live) so.load_node(nd, le, n);
    T phi{}, U{}, V{};
    schur_solve_with<P, EPB, A>(sm, g, e, le, n, live, nd, [&](int m) { return so.srow(le, n, m); }, EG, x0, xU, xV,
                                phi, U, V);
    if (live) {
        Z[o] = A::to(phi);
        Z[fs + o] = A::to(U);
        Z[2 * fs + o] = A::to(V);
    }
}

template <int P, int EPB, class A>
__global__ void __launch_bounds__(EPB * P * P)
    schur_recover_staged_kernel(Geom g, const typename A::T* __restrict__ S, const typename A::T* __restrict__ aux,
                                const typename A::T* __restrict__ EG, const double* __restrict__ Z,
                                const double* __restrict__ R1, const double* __restrict__ tau_edge,
                                const double* __restrict__ qhat, double beta, double inv_aii, double* __restrict__ Q,
                                double* __restrict__ Lst, unsigned* err, float* __restrict__ Q32) {
    using T = typename A::T;
    constexpr int Np = P * P, NF = 3 * P;
    __shared__ SchurSmem<P, EPB, A> sm;
    __shared__ StagedOps<P, EPB, A> so;
    const int le = threadIdx.x / Np, n = threadIdx.x % Np, i = n % P, j = n / P;
    const int e0 = blockIdx.x * EPB, e = e0 + le;
    const int ne = g.n_el - e0 < EPB ? g.n_el - e0 : EPB;
    const bool live = le < EPB && e < g.n_el;
    so.issue(S, aux, e0, ne);
    const size_t fs = (size_t)g.n_el * Np, o = (size_t)e * Np + n;
    double u[3] = {0.0, 0.0, 0.0}, zv[3] = {0.0, 0.0, 0.0}, rv[3] = {0.0, 0.0, 0.0};
    if (live) {
        for (int c = 0; c < 3; ++c) {
            zv[c] = Z[c * fs + o];
            rv[c] = R1[c * fs + o];
        }
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && i == 0) || (f == 1 && i == P - 1) || (f == 2 && j == 0) ||
                            (f == 3 && j == P - 1);
            if (!on) continue;
            const int b = (f < 2) ? j : i;
            const int ed = edge_of_face(e, f, g);
            const double tau = tau_edge[(size_t)ed * P + b];
            for (int c = 0; c < 3; ++c) u[c] += tau * qhat[(size_t)ed * NF + c * P + b];
        }
    }
    if (!so.wait(err)) return;
    SchurNode<A> nd;
    if (live) so.load_node(nd, le, n);
    T y[3];
    schur_solve_with<P, EPB, A>(sm, g, e, le, n, live, nd, [&](int m) { return so.srow(le, n, m); }, EG,
                                A::from(u[0]), A::from(u[1]), A::from(u[2]), y[0], y[1], y[2]);
    if (live) {
        const double kk = beta * dt_factor(g, e);
        for (int c = 0; c < 3; ++c) {
            const size_t oc = c * fs + o;
            const double q = zv[c] + kk * A::to(y[c]);
            if (Q32) Q32[oc] = f64_to_f32(q);
            else Q[oc] = q;
            Lst[oc] = q - rv[c];
        }
    }
}

// Tiles of the Schur-complement kernels: elements per block for about 256 (tile 0, the default),
// 128 or 512 threads; the autotuner tries them at create for degrees 2..4.  Tile 3 (degree 3):
// 128 threads with the operators staged in shared memory.
constexpr int schur_tile_threads(int t) { return t == 1 || t == 3 ? 128 : t == 2 ? 512 : 256; }
template <int P>
constexpr int schur_epb_for(int threads) {
    return threads / (P * P) > 0 ? threads / (P * P) : 1;
}

template <int P, class A, int TILE>
void schur_condense_t(const Geom& g, const LocalOps& ops, const double* R1, double* Z, cudaStream_t s,
                      const R1Source& src) {
    using T = typename A::T;
    constexpr int EPB = schur_epb_for<P>(schur_tile_threads(TILE));
    schur_condense_kernel<P, EPB, A><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(
        g, static_cast<const T*>(ops.S), static_cast<const T*>(ops.aux), static_cast<const T*>(ops.EG), R1, Z, src);
    count_launches(1);
}

template <int P, class A, int TILE>
void schur_recover_t(const Geom& g, const LocalOps& ops, const double* Z, const double* R1, const double* tau_edge,
                     const double* qhat, double beta, double inv_aii, double* Q, double* Lst, cudaStream_t s,
                     float* Q32) {
    using T = typename A::T;
    constexpr int EPB = schur_epb_for<P>(schur_tile_threads(TILE));
    schur_recover_kernel<P, EPB, A><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(
        g, static_cast<const T*>(ops.S), static_cast<const T*>(ops.aux), static_cast<const T*>(ops.EG), Z, R1,
        tau_edge, qhat, beta, inv_aii, Q, Lst, Q32);
    count_launches(1);
}

template <int P, class A>
constexpr bool schur_staged_ok() {
    return P == 4 && StagedOps<P, schur_epb_for<P>(128), A>::kFits;
}

template <int P, class A>
void schur_condense(const Geom& g, const LocalOps& ops, const double* R1, double* Z, cudaStream_t s,
                    const R1Source& src = R1Source{}) {
    if constexpr (schur_staged_ok<P, A>()) {
        if (ops.schur_tile_c == 3) {
            using T = typename A::T;
            constexpr int EPB = schur_epb_for<P>(128);
            schur_condense_staged_kernel<P, EPB, A><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(
                g, static_cast<const T*>(ops.S), static_cast<const T*>(ops.aux), static_cast<const T*>(ops.EG), R1, Z,
                reinterpret_cast<unsigned*>(ops.error), src);
            count_launches(1);
            return;
        }
    }
    if constexpr (P >= 3 && P <= 5) {
        if (ops.schur_tile_c == 1) return schur_condense_t<P, A, 1>(g, ops, R1, Z, s, src);
        if (ops.schur_tile_c == 2) return schur_condense_t<P, A, 2>(g, ops, R1, Z, s, src);
    }
    schur_condense_t<P, A, 0>(g, ops, R1, Z, s, src);
}

template <int P, class A>
void schur_recover(const Geom& g, const LocalOps& ops, const double* Z, const double* R1, const double* tau_edge,
                   const double* qhat, double beta, double inv_aii, double* Q, double* Lst, cudaStream_t s,
                   float* Q32 = nullptr) {
    if constexpr (schur_staged_ok<P, A>()) {
        if (ops.schur_tile_r == 3) {
            using T = typename A::T;
            constexpr int EPB = schur_epb_for<P>(128);
            schur_recover_staged_kernel<P, EPB, A><<<(g.n_el + EPB - 1) / EPB, EPB * P * P, 0, s>>>(
                g, static_cast<const T*>(ops.S), static_cast<const T*>(ops.aux), static_cast<const T*>(ops.EG), Z, R1,
                tau_edge, qhat, beta, inv_aii, Q, Lst, reinterpret_cast<unsigned*>(ops.error), Q32);
            count_launches(1);
            return;
        }
    }
    if constexpr (P >= 3 && P <= 5) {
        if (ops.schur_tile_r == 1)
            return schur_recover_t<P, A, 1>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32);
        if (ops.schur_tile_r == 2)
            return schur_recover_t<P, A, 2>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32);
    }
    schur_recover_t<P, A, 0>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32);
}

// Time each tile of the Schur condensation and recovery (two warm-up and five timed launches
// each, CUDA events) on the handle's operators and keep the fastest of each in ops.
template <int P, class A>
cudaError_t autotune_schur(const Geom& g, LocalOps& ops, double* R1, double* Z, const double* tau_edge,
                           const double* qhat, double* Q, double* Lst, cudaStream_t s) {
    if constexpr (P < 3 || P > 5) {
        return cudaSuccess;
    } else {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return cudaGetLastError();
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return cudaGetLastError();
        }
        float best_c = 1e30f, best_r = 1e30f;
        int tc = 0, tr = 0;
        cudaError_t err = cudaSuccess;
        const int n_tiles = schur_staged_ok<P, A>() ? 4 : 3;
        for (int t = 0; t < n_tiles && err == cudaSuccess; ++t) {
            ops.schur_tile_c = ops.schur_tile_r = t;
            float ms_c = 0.f, ms_r = 0.f;
            for (int k = 0; k < 2; ++k) schur_condense<P, A>(g, ops, R1, Z, s);
            cudaEventRecord(a, s);
            for (int k = 0; k < 5; ++k) schur_condense<P, A>(g, ops, R1, Z, s);
            cudaEventRecord(b, s);
            err = cudaEventSynchronize(b);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_c, a, b);
            for (int k = 0; k < 2; ++k) schur_recover<P, A>(g, ops, Z, R1, tau_edge, qhat, 1.0, 1.0, Q, Lst, s);
            cudaEventRecord(a, s);
            for (int k = 0; k < 5; ++k) schur_recover<P, A>(g, ops, Z, R1, tau_edge, qhat, 1.0, 1.0, Q, Lst, s);
            cudaEventRecord(b, s);
            if (err == cudaSuccess) err = cudaEventSynchronize(b);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_r, a, b);
            if (err == cudaSuccess && ms_c < best_c) { best_c = ms_c; tc = t; }
            if (err == cudaSuccess && ms_r < best_r) { best_r = ms_r; tr = t; }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        ops.schur_tile_c = tc;
        ops.schur_tile_r = tr;
        ops.tile_condense = schur_epb_for<P>(schur_tile_threads(tc));
        ops.tile_recover = schur_epb_for<P>(schur_tile_threads(tr));
        if (err == cudaSuccess) err = cudaGetLastError();
        return err;
    }
}

template <int P, class A>
cudaError_t schur_setup(const Geom& g, const double* Ainv, const double* phiB, const double* tau_edge, double dta,
                        void* S, void* aux, void* EG, cudaStream_t s) {
    using T = typename A::T;
    const size_t n = (size_t)g.n_el * g.Np;
    schur_setup_kernel<P, A><<<(int)((n + 255) / 256), 256, 0, s>>>(g, Ainv, phiB, tau_edge, dta,
                                                                     static_cast<T*>(S), static_cast<T*>(aux));
    const int ne = g.batch * 2 * P * P;
    schur_eg_kernel<P, A><<<(ne + 255) / 256, 256, 0, s>>>(g, dta, static_cast<T*>(EG));
    count_launches(2);
    return cudaGetLastError();
}

template <int P>
cudaError_t build_local_launch(const Geom& g, const double* phiB, const double* tau_edge, double dta,
                               double* Ainv, double* Se, int* singular, cudaStream_t s) {
    constexpr int NV = 3 * P * P;
    constexpr bool kGmem = (size_t)NV * 2 * NV * sizeof(double) > 200 * 1024;
    const size_t small = (size_t)(P * P + 4 * P) * sizeof(double);
    const size_t smem = kGmem ? small : (size_t)NV * 2 * NV * sizeof(double) + small;
    cudaError_t err = cudaFuncSetAttribute(build_local_kernel<P, kGmem>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (!kGmem) {
        build_local_kernel<P, false><<<g.n_el, 128, smem, s>>>(g, phiB, tau_edge, dta, Ainv, Se, singular, 0,
                                                               nullptr);
        count_launches(1);
        return cudaGetLastError();
    }
    // global workspace: chunks of at most 512 elements (NV = 243 at k = 8: 0.9 MB per element)
    const int chunk = g.n_el < 512 ? g.n_el : 512;
    double* work = nullptr;
    err = cudaMallocAsync(&work, (size_t)chunk * NV * 2 * NV * sizeof(double), s);
    if (err != cudaSuccess) return err;
    for (int e0 = 0; e0 < g.n_el; e0 += chunk) {
        const int n = g.n_el - e0 < chunk ? g.n_el - e0 : chunk;
        build_local_kernel<P, true><<<n, 256, smem, s>>>(g, phiB, tau_edge, dta, Ainv, Se, singular, e0, work);
        count_launches(1);
    }
    err = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(work, s);
    return err != cudaSuccess ? err : e2;
}

template <int P>
cudaError_t assemble_launch(const Geom& g, const double* Se, double* S7, double* Srr, double* Minv,
                            double* Stil, int* Scol, int* singular, cudaStream_t s) {
    gather_rows_kernel<P><<<g.n_edges, 128, 0, s>>>(g, Se, S7, Srr, Scol);
    count_launches(1);
    invert_diag_kernel<P><<<g.n_edges, 64, 0, s>>>(S7, Minv, singular);
    count_launches(1);
    precondition_kernel<P><<<g.n_edges, 128, 0, s>>>(g.n_edges, S7, Minv, Scol, Stil);
    count_launches(1);
    return cudaGetLastError();
}

// Tiles (elements per block) of the FP32-pair local kernels: index 0 is 256 / NV, then 1, 2, 4, 8
// where the block stays within 1024 threads.
template <int P>
constexpr int tile_epb(int t) {
    constexpr int NV = 3 * P * P;
    const int e = t == 0 ? (256 / NV > 0 ? 256 / NV : 1) : (1 << (t - 1));
    return e * NV <= 1024 ? e : 0;
}

template <int P, int EPB>
void x2_apply(const Geom& g, const LocalOps& ops, const double* R1, double* Z, cudaStream_t s) {
    constexpr int NV = 3 * P * P;
    if constexpr (EPB > 0 && EPB * NV <= 1024) {
        apply_ainv_x2_kernel<P, EPB><<<(g.n_el + EPB - 1) / EPB, EPB * NV, 0, s>>>(g, ops.Ahi, ops.Alo, R1, Z);
        count_launches(1);
    }
}

template <int P, int EPB>
void x2_recover(const Geom& g, const LocalOps& ops, const double* Z, const double* R1, const double* tau_edge,
                const double* qhat, double beta, double inv_aii, double* Q, double* Lst, cudaStream_t s) {
    constexpr int NV = 3 * P * P;
    if constexpr (EPB > 0 && EPB * NV <= 1024) {
        recover_x2_kernel<P, EPB><<<(g.n_el + EPB - 1) / EPB, EPB * NV, 0, s>>>(g, ops.Ahi, ops.Alo, Z, R1, tau_edge,
                                                                              qhat, beta, inv_aii, Q, Lst);
        count_launches(1);
    }
}

template <int P>
void x2_apply_tile(int t, const Geom& g, const LocalOps& ops, const double* R1, double* Z, cudaStream_t s) {
    switch (t) {
        case 1: return x2_apply<P, tile_epb<P>(1)>(g, ops, R1, Z, s);
        case 2: return x2_apply<P, tile_epb<P>(2)>(g, ops, R1, Z, s);
        case 3: return x2_apply<P, tile_epb<P>(3)>(g, ops, R1, Z, s);
        case 4: return x2_apply<P, tile_epb<P>(4)>(g, ops, R1, Z, s);
        default: return x2_apply<P, tile_epb<P>(0)>(g, ops, R1, Z, s);
    }
}

template <int P>
void x2_recover_tile(int t, const Geom& g, const LocalOps& ops, const double* Z, const double* R1,
                     const double* tau_edge, const double* qhat, double beta, double inv_aii, double* Q, double* Lst,
                     cudaStream_t s) {
    switch (t) {
        case 1: return x2_recover<P, tile_epb<P>(1)>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
        case 2: return x2_recover<P, tile_epb<P>(2)>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
        case 3: return x2_recover<P, tile_epb<P>(3)>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
        case 4: return x2_recover<P, tile_epb<P>(4)>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
        default: return x2_recover<P, tile_epb<P>(0)>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
    }
}

// Time every valid tile of both FP32-pair kernels on the handle's own operators (one warm-up and
// three timed launches each, CUDA events on the stream) and keep the fastest in ops.
template <int P>
cudaError_t autotune_x2(const Geom& g, LocalOps& ops, double* R1, double* Z, const double* tau_edge,
                        const double* qhat, double* Q, double* Lst, cudaStream_t s) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return cudaGetLastError();
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return cudaGetLastError();
    }
    float best_c = 1e30f, best_r = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int t = 0; t < 5 && err == cudaSuccess; ++t) {
        if (tile_epb<P>(t) == 0 || (t > 0 && tile_epb<P>(t) == tile_epb<P>(0))) continue;
        float ms_c = 0.f, ms_r = 0.f;
        x2_apply_tile<P>(t, g, ops, R1, Z, s);
        cudaEventRecord(a, s);
        for (int k = 0; k < 3; ++k) x2_apply_tile<P>(t, g, ops, R1, Z, s);
        cudaEventRecord(b, s);
        err = cudaEventSynchronize(b);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_c, a, b);
        x2_recover_tile<P>(t, g, ops, Z, R1, tau_edge, qhat, 1.0, 1.0, Q, Lst, s);
        cudaEventRecord(a, s);
        for (int k = 0; k < 3; ++k) x2_recover_tile<P>(t, g, ops, Z, R1, tau_edge, qhat, 1.0, 1.0, Q, Lst, s);
        cudaEventRecord(b, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_r, a, b);
        if (err == cudaSuccess && ms_c < best_c) { best_c = ms_c; ops.tile_condense = tile_epb<P>(t); ops.tile_condense_index = t; }
        if (err == cudaSuccess && ms_r < best_r) { best_r = ms_r; ops.tile_recover = tile_epb<P>(t); ops.tile_recover_index = t; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (err == cudaSuccess) err = cudaGetLastError();
    return err;
}

template <int P>
cudaError_t condense_launch(const Geom& g, const LocalOps& ops, const double* R1, const double* phiB,
                            const double* tau_edge, double* Z, double* gvec, cudaStream_t s, double t,
                            const R1Source* src) {
    constexpr int NV = 3 * P * P;
    constexpr int EPB = (256 / NV) > 0 ? 256 / NV : 1;
    const int blocks = (g.n_el + EPB - 1) / EPB;
    if (src && src->base && !ops.schur) {   // the other kernels read R1 as it stands: form it first
        const cudaError_t e = launch_combine((size_t)3 * g.n_el * g.Np, src->base, src->t, const_cast<double*>(R1),
                                             nullptr, s);
        if (e != cudaSuccess) return e;
    }
    const R1Source none{};
    if (ops.schur) {
        const R1Source& rs = src ? *src : none;
        if (ops.kind == 3) schur_condense<P, ArithF2>(g, ops, R1, Z, s, rs);
        else schur_condense<P, ArithF64>(g, ops, R1, Z, s, rs);
    } else if (ops.kind == 2 || ops.kind == 4) {
        cudaError_t e = ops.kind == 2 ? launch_local_tc(g, 0, ops.image, R1, nullptr, nullptr, nullptr, 0.0, 0.0, Z,
                                                        nullptr, ops.error, s)
                                      : launch_local_tc_split(g, 0, ops.image, R1, nullptr, nullptr, nullptr, 0.0,
                                                              0.0, Z, nullptr, ops.error, s);
        if (e != cudaSuccess) return e;
    } else if (ops.kind == 3) {
        x2_apply_tile<P>(ops.tile_condense_index, g, ops, R1, Z, s);
    } else if (ops.kind == 1) {
        apply_ainv_kernel<P, float><<<blocks, EPB * NV, 0, s>>>(g, ops.Ainv32, R1, Z);
        count_launches(1);
    } else {
        apply_ainv_kernel<P, double><<<blocks, EPB * NV, 0, s>>>(g, ops.Ainv, R1, Z);
        count_launches(1);
    }
    const int n = g.n_edges * P;
    edge_rhs_kernel<P><<<(n + 255) / 256, 256, 0, s>>>(g, Z, phiB, tau_edge, gvec, t);
    count_launches(1);
    return cudaGetLastError();
}

template <int P>
cudaError_t recover_launch(const Geom& g, const LocalOps& ops, const double* Z, const double* R1,
                           const double* tau_edge, const double* qhat, double beta, double inv_aii,
                           double* Q, double* Lst, cudaStream_t s, float* Q32) {
    constexpr int NV = 3 * P * P;
    constexpr int EPB = (256 / NV) > 0 ? 256 / NV : 1;
    const int blocks = (g.n_el + EPB - 1) / EPB;
    if (ops.schur) {
        if (inv_aii != 1.0) return cudaErrorInvalidValue;   // the Schur kernels write Q - R1
        if (ops.kind == 3) schur_recover<P, ArithF2>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32);
        else schur_recover<P, ArithF64>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32);
        return cudaGetLastError();
    }
    if (Q32) return cudaErrorInvalidValue;   // the FP32 stage output is the Schur kernels' only
    if (ops.kind == 2)
        return launch_local_tc(g, 1, ops.image, R1, Z, tau_edge, qhat, beta, inv_aii, Q, Lst, ops.error, s);
    if (ops.kind == 4)
        return launch_local_tc_split(g, 1, ops.image, R1, Z, tau_edge, qhat, beta, inv_aii, Q, Lst, ops.error, s);
    if (ops.kind == 3) {
        x2_recover_tile<P>(ops.tile_recover_index, g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s);
        return cudaGetLastError();
    }
    if (ops.kind == 1)
        recover_kernel<P, float><<<blocks, EPB * NV, 0, s>>>(g, ops.Ainv32, Z, R1, tau_edge, qhat, beta,
                                                             inv_aii, Q, Lst);
    else
        recover_kernel<P, double><<<blocks, EPB * NV, 0, s>>>(g, ops.Ainv, Z, R1, tau_edge, qhat, beta,
                                                              inv_aii, Q, Lst);
    count_launches(1);
    return cudaGetLastError();
}

// ---- ensembles: condensation and recovery of every group in one persistent launch each ------------
template <int P>
__host__ __device__ constexpr int ens_schur_epb() {
    return 256 / (P * P);
}

__global__ void __launch_bounds__(256) ens_condense_kernel(EnsTable t, const double* __restrict__ R1,
                                                           double* __restrict__ Z) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        using T = float2;
        const T* S = static_cast<const T*>(G.S2);
        const T* aux = static_cast<const T*>(G.aux2);
        const T* EG = static_cast<const T*>(G.EG2);
        switch (G.g.P) {
            case 3: schur_condense_body<3, ens_schur_epb<3>(), ArithF2>(bid, G.g, S, aux, EG, R1 + G.off3, Z + G.off3); break;
            case 4: schur_condense_body<4, ens_schur_epb<4>(), ArithF2>(bid, G.g, S, aux, EG, R1 + G.off3, Z + G.off3); break;
            case 5: schur_condense_body<5, ens_schur_epb<5>(), ArithF2>(bid, G.g, S, aux, EG, R1 + G.off3, Z + G.off3); break;
            default: break;
        }
    });
}

__global__ void __launch_bounds__(256) ens_edge_rhs_kernel(EnsTable t, const double* __restrict__ Z,
                                                           double* __restrict__ gvec) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        switch (G.g.P) {
            case 3: edge_rhs_body<3>(bid, G.g, Z + G.off3, G.phiB, G.tau, gvec + G.offt, 0.0); break;
            case 4: edge_rhs_body<4>(bid, G.g, Z + G.off3, G.phiB, G.tau, gvec + G.offt, 0.0); break;
            case 5: edge_rhs_body<5>(bid, G.g, Z + G.off3, G.phiB, G.tau, gvec + G.offt, 0.0); break;
            default: break;
        }
    });
}

__global__ void __launch_bounds__(256) ens_recover_kernel(EnsTable t, const double* __restrict__ Z,
                                                          const double* __restrict__ R1, const double* __restrict__ qhat,
                                                          double inv_aii, double* __restrict__ Q, double* __restrict__ Lst) {
    ens_walk(t, [&](const EnsGroup& G, int bid) {
        using T = float2;
        const T* S = static_cast<const T*>(G.S2);
        const T* aux = static_cast<const T*>(G.aux2);
        const T* EG = static_cast<const T*>(G.EG2);
        const size_t o = G.off3, ot = G.offt;
        switch (G.g.P) {
            case 3: schur_recover_body<3, ens_schur_epb<3>(), ArithF2>(bid, G.g, S, aux, EG, Z + o, R1 + o, G.tau, qhat + ot, G.beta, inv_aii, Q + o, Lst + o); break;
            case 4: schur_recover_body<4, ens_schur_epb<4>(), ArithF2>(bid, G.g, S, aux, EG, Z + o, R1 + o, G.tau, qhat + ot, G.beta, inv_aii, Q + o, Lst + o); break;
            case 5: schur_recover_body<5, ens_schur_epb<5>(), ArithF2>(bid, G.g, S, aux, EG, Z + o, R1 + o, G.tau, qhat + ot, G.beta, inv_aii, Q + o, Lst + o); break;
            default: break;
        }
    });
}

int ens_elem_blocks(const EnsGroup& G) {
    const int epb = 256 / G.g.Np;
    return (G.g.n_el + epb - 1) / epb;
}

}  // namespace

bool schur_tile_ready(int P, bool pairs, int t) {
    if (t == 0) return true;
    if (P < 3 || P > 5 || t < 0) return false;
    if (t < 3) return true;
    return t == 3 && (pairs ? schur_staged_ok<4, ArithF2>() : schur_staged_ok<4, ArithF64>()) && P == 4;
}

int schur_tile_epb(int P, int t) {
    const int th = schur_tile_threads(t);
    return th / (P * P) > 0 ? th / (P * P) : 1;
}


cudaError_t launch_ens_condense(const EnsHost& E, const double* R1, double* Z, double* gvec, cudaStream_t s) {
    const EnsTable te = ens_table(E, ens_elem_blocks);
    const EnsTable tr = ens_table(E, [](const EnsGroup& G) { return (G.g.n_edges * G.g.P + 255) / 256; });
    ens_condense_kernel<<<ens_grid(ens_condense_kernel, te.start[te.ngroups]), 256, 0, s>>>(te, R1, Z);
    ens_edge_rhs_kernel<<<ens_grid(ens_edge_rhs_kernel, tr.start[tr.ngroups]), 256, 0, s>>>(tr, Z, gvec);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_ens_recover(const EnsHost& E, const double* Z, const double* R1, const double* qhat,
                               double inv_aii, double* Q, double* Lst, cudaStream_t s) {
    if (inv_aii != 1.0) return cudaErrorInvalidValue;   // the Schur kernels write Q - R1
    const EnsTable te = ens_table(E, ens_elem_blocks);
    ens_recover_kernel<<<ens_grid(ens_recover_kernel, te.start[te.ngroups]), 256, 0, s>>>(te, Z, R1, qhat, inv_aii, Q,
                                                                                          Lst);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_autotune_local(const Geom& g, LocalOps& ops, double* R1, double* Z, const double* tau_edge,
                                  const double* qhat, double* Q, double* Lst, cudaStream_t s) {
    if (ops.schur) {
#define SCALL(P)                                                                                  \
    return ops.kind == 3 ? autotune_schur<P, ArithF2>(g, ops, R1, Z, tau_edge, qhat, Q, Lst, s)   \
                         : autotune_schur<P, ArithF64>(g, ops, R1, Z, tau_edge, qhat, Q, Lst, s)
        switch (g.P) {
            case 3: SCALL(3);
            case 4: SCALL(4);
            case 5: SCALL(5);
            default: return cudaSuccess;
        }
#undef SCALL
    }
    if (ops.kind != 3) return cudaSuccess;
#define CALL(P) autotune_x2<P>(g, ops, R1, Z, tau_edge, qhat, Q, Lst, s)
    switch (g.P) {
        case 2: return CALL(2);
        case 3: return CALL(3);
        case 4: return CALL(4);
        case 5: return CALL(5);
        case 6: return CALL(6);
        case 7: return CALL(7);
        case 8: return CALL(8);
        case 9: return CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_schur_setup(const Geom& g, const double* Ainv, const double* phiB, const double* tau_edge,
                               double dta, bool f32x2, void* S, void* aux, void* EG, cudaStream_t s) {
#define CALL(P)                                                                                      \
    return f32x2 ? schur_setup<P, ArithF2>(g, Ainv, phiB, tau_edge, dta, S, aux, EG, s)              \
                 : schur_setup<P, ArithF64>(g, Ainv, phiB, tau_edge, dta, S, aux, EG, s)
    switch (g.P) {
        case 2: CALL(2);
        case 3: CALL(3);
        case 4: CALL(4);
        case 5: CALL(5);
        case 6: CALL(6);
        case 7: CALL(7);
        case 8: CALL(8);
        case 9: CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_split_f32x2(const double* a, float* hi, float* lo, size_t n, cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, 0, s>>>(a, hi, lo, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_build_local(const Geom& g, const double* phiB, const double* tau_edge, double dta,
                               double* Ainv, double* Se, int* singular, cudaStream_t s) {
#define CALL(P) build_local_launch<P>(g, phiB, tau_edge, dta, Ainv, Se, singular, s)
    switch (g.P) {
        case 2: return CALL(2);
        case 3: return CALL(3);
        case 4: return CALL(4);
        case 5: return CALL(5);
        case 6: return CALL(6);
        case 7: return CALL(7);
        case 8: return CALL(8);
        case 9: return CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_assemble_trace(const Geom& g, const double* Se, double* S7, double* Srr,
                                  double* Minv, double* Stil, int* Scol, int* singular,
                                  cudaStream_t s) {
#define CALL(P) assemble_launch<P>(g, Se, S7, Srr, Minv, Stil, Scol, singular, s)
    switch (g.P) {
        case 2: return CALL(2);
        case 3: return CALL(3);
        case 4: return CALL(4);
        case 5: return CALL(5);
        case 6: return CALL(6);
        case 7: return CALL(7);
        case 8: return CALL(8);
        case 9: return CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_condense(const Geom& g, const LocalOps& ops, const double* R1, const double* phiB,
                            const double* tau_edge, double* Z, double* gvec, cudaStream_t s, double t,
                            const R1Source* src) {
    if (src && src->base && (src->t.n < 0 || src->t.n > kR1FusedTerms)) return cudaErrorInvalidValue;
#define CALL(P) condense_launch<P>(g, ops, R1, phiB, tau_edge, Z, gvec, s, t, src)
    switch (g.P) {
        case 2: return CALL(2);
        case 3: return CALL(3);
        case 4: return CALL(4);
        case 5: return CALL(5);
        case 6: return CALL(6);
        case 7: return CALL(7);
        case 8: return CALL(8);
        case 9: return CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_recover(const Geom& g, const LocalOps& ops, const double* Z, const double* R1,
                           const double* tau_edge, const double* qhat, double beta, double inv_aii,
                           double* Q, double* Lst, cudaStream_t s, float* Q32) {
#define CALL(P) recover_launch<P>(g, ops, Z, R1, tau_edge, qhat, beta, inv_aii, Q, Lst, s, Q32)
    switch (g.P) {
        case 2: return CALL(2);
        case 3: return CALL(3);
        case 4: return CALL(4);
        case 5: return CALL(5);
        case 6: return CALL(6);
        case 7: return CALL(7);
        case 8: return CALL(8);
        case 9: return CALL(9);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace hdgdg
