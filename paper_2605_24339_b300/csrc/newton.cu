// newton.cu -- kernels of the implicit-Euler time step: compressible
// Neo-Hookean tets, deterministic assembly of the gradient and of the global
// block-sparse (3x3) Hessian, block-Jacobi preconditioned CG, and the
// energies the backtracking line search compares.
//
// The step minimises E(x) = 1/2 (x - xhat)^T M (x - xhat) + h^2 (Psi_NH(x) +
// Psi_GMCP(x)) over the free vertices (paper Sec. 2.1 problem statement;
// contact potential of Sec. 4.2).  Elasticity (not specified by the paper):
//   Psi = V [ mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2 ],  F = Ds Dm^-1
// with dP/dF (9x9, vec index 3 i + j) projected onto the PSD cone by a cyclic
// Jacobi eigen-decomposition and mapped to the 12x12 tet block by dF/dx.
//
// Every sum over tets, vertices or blocks is a gather in a fixed order or a
// fixed-shape tree reduction, so results do not depend on scheduling.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <memory>
#include <vector>

#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

__device__ __forceinline__ double det3(const double* A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
__device__ __forceinline__ void inv3(const double* A, double* I) {
    const double d = det3(A);
    I[0] = (A[4] * A[8] - A[5] * A[7]) / d; I[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    I[2] = (A[1] * A[5] - A[2] * A[4]) / d; I[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    I[4] = (A[0] * A[8] - A[2] * A[6]) / d; I[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    I[6] = (A[3] * A[7] - A[4] * A[6]) / d; I[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    I[8] = (A[0] * A[4] - A[1] * A[3]) / d;
}

// (J - 1) - ln J without cancellation: Taylor series for |d| < 1e-2
// (truncation below 1e-17 relative), else the plain difference
__device__ __forceinline__ double d_minus_log1p(double d) {
    if (fabs(d) < 1e-2)
        return d * d * (1.0 / 2 - d * (1.0 / 3 - d * (1.0 / 4 - d * (1.0 / 5 - d * (1.0 / 6 - d * (1.0 / 7 - d * (1.0 / 8 - d / 9.0)))))));
    return d - log1p(d);
}

struct ElasticView {
    int64_t nt;
    const int32_t* tets;   // [nt][4]
    const double* Dminv;   // [nt][9]
    const double* vol;     // [nt]
    const double* X;       // rest positions [nv][3]
    double mu, lam;
};

// Displacement gradient H = (Ds - Dm) Dm^-1 from the vertex displacements
// u = x - X, F = I + H, and the Neo-Hookean energy of the tet in the form
//   V [mu ((J-1) - ln J - q) + mu/2 |H|^2 + lambda/2 (ln J)^2],
//   J - 1 = tr H + q, q = sum of principal 2x2 minors of H + det H,
// (algebraically mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2, with the
// first-order terms cancelled exactly so the energy keeps its relative
// precision at small strain).  Returns false if J <= 0.
__device__ __forceinline__ bool nh_energy(const double* Dmi, double vol, double mu, double lam,
                                          const double* x4, const double* X4, double* psi, double* F,
                                          double* lnJ) {
    double Du[9], H[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Du[3 * r + c] = (x4[3 * (c + 1) + r] - X4[3 * (c + 1) + r]) - (x4[r] - X4[r]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            H[3 * i + j] = Du[3 * i] * Dmi[j] + Du[3 * i + 1] * Dmi[3 + j] + Du[3 * i + 2] * Dmi[6 + j];
    for (int i = 0; i < 9; ++i) F[i] = H[i];
    F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
    const double trH = H[0] + H[4] + H[8];
    const double minors = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
    const double q = minors + det3(H);
    const double jm1 = trH + q;
    if (!(jm1 > -1.0)) return false;
    double nH = 0.0;
    for (int i = 0; i < 9; ++i) nH += H[i] * H[i];
    *lnJ = log1p(jm1);
    *psi = vol * (mu * (d_minus_log1p(jm1) - q) + 0.5 * mu * nH + 0.5 * lam * (*lnJ) * (*lnJ));
    return true;
}

__device__ __forceinline__ void load_tet(const ElasticView& E, const double* x, int64_t t, double* x4) {
    for (int a = 0; a < 4; ++a) {
        const int64_t v = E.tets[4 * t + a];
        x4[3 * a] = x[3 * v]; x4[3 * a + 1] = x[3 * v + 1]; x4[3 * a + 2] = x[3 * v + 2];
    }
}

// cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (row-major,
// in registers); on return A's diagonal holds the eigenvalues and V's
// columns the eigenvectors
__device__ __forceinline__ void jacobi3(double* A, double* V) {
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
#pragma unroll 1
    for (int sweep = 0; sweep < 32; ++sweep) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double tot = off + 0.5 * (A[0] * A[0] + A[4] * A[4] + A[8] * A[8]);
        if (off <= 1e-33 * tot || off == 0.0) break;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2;
            const double apq = A[3 * p + q];
            if (apq == 0.0) continue;
            const double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double arp = A[3 * r + p], arq = A[3 * r + q];
                A[3 * r + p] = c * arp - s * arq;
                A[3 * r + q] = s * arp + c * arq;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double apr = A[3 * p + r], aqr = A[3 * q + r];
                A[3 * p + r] = c * apr - s * aqr;
                A[3 * q + r] = s * apr + c * aqr;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double vrp = V[3 * r + p], vrq = V[3 * r + q];
                V[3 * r + p] = c * vrp - s * vrq;
                V[3 * r + q] = s * vrp + c * vrq;
            }
        }
    }
}

// PSD-projected Neo-Hookean Hessian of one tet, written as its 4x4 blocks
// of 3x3.  dP/dF of an isotropic energy has a closed-form eigensystem in the
// singular values of F = U diag(s) V^T (Smith, de Goes, Kim 2019, "Analytic
// eigensystems for isotropic distortion energies"); for this energy, with
// c = mu - lambda ln J:
//   twist modes U (e_i e_j^T - e_j e_i^T) V^T / sqrt 2:  mu - c / (s_i s_j)
//   flip modes  U (e_i e_j^T + e_j e_i^T) V^T / sqrt 2:  mu + c / (s_i s_j)
//   scaling modes U diag(e) V^T, e the eigenvectors of the 3x3
//     A_ii = mu + (c + lambda) / s_i^2, A_ij = lambda / (s_i s_j).
// Clamping the eigenvalues at zero gives the same (unique) projection as a
// 9x9 eigen-decomposition.  With D[m] the rows of dF/dx and d_m = V^T D[m],
// block (m, n) = V_tet U M_mn U^T, M_mn = sum_k max(l_k, 0) (E_k d_m)(E_k d_n)^T.
__device__ void nh_hessian_blocks(const double* F, double lnJ, double mu, double lam, const double* D,
                                  double vol, double* out /* [144] */) {
    // SVD from the eigen-decomposition of F^T F
    double S[9], V[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    jacobi3(S, V);
    const double detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                        V[2] * (V[3] * V[7] - V[4] * V[6]);
    if (detV < 0.0) { V[2] = -V[2]; V[5] = -V[5]; V[8] = -V[8]; }
    double B[9];   // F V, columns b_k
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) B[3 * i + k] = F[3 * i] * V[k] + F[3 * i + 1] * V[3 + k] + F[3 * i + 2] * V[6 + k];
    double U[9], sg[3];
    {
        double n0 = sqrt(B[0] * B[0] + B[3] * B[3] + B[6] * B[6]);
        double u0[3] = {B[0] / n0, B[3] / n0, B[6] / n0};
        double pr = u0[0] * B[1] + u0[1] * B[4] + u0[2] * B[7];
        double w1[3] = {B[1] - pr * u0[0], B[4] - pr * u0[1], B[7] - pr * u0[2]};
        double n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
        double u1[3];
        if (n1 > 1e-300) {
            u1[0] = w1[0] / n1; u1[1] = w1[1] / n1; u1[2] = w1[2] / n1;
        } else {   // any unit vector orthogonal to u0
            const double ax = fabs(u0[0]), ay = fabs(u0[1]), az = fabs(u0[2]);
            double e[3] = {0, 0, 0};
            e[(ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2)] = 1.0;
            const double d = e[0] * u0[0] + e[1] * u0[1] + e[2] * u0[2];
            double w[3] = {e[0] - d * u0[0], e[1] - d * u0[1], e[2] - d * u0[2]};
            const double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            u1[0] = w[0] / nw; u1[1] = w[1] / nw; u1[2] = w[2] / nw;
        }
        double u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
        sg[0] = n0;
        sg[1] = u1[0] * B[1] + u1[1] * B[4] + u1[2] * B[7];
        sg[2] = u2[0] * B[2] + u2[1] * B[5] + u2[2] * B[8];
        for (int i = 0; i < 3; ++i) { U[3 * i] = u0[i]; U[3 * i + 1] = u1[i]; U[3 * i + 2] = u2[i]; }
    }
    const double c = mu - lam * lnJ;
    // scaling block and its projection
    double A[9], W[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = (i == j) ? mu + (c + lam) / (sg[i] * sg[i]) : lam / (sg[i] * sg[j]);
    jacobi3(A, W);
    double Ah[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double sum = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double l = A[4 * k];
                if (l > 0.0) sum += W[3 * i + k] * l * W[3 * j + k];
            }
            Ah[3 * i + j] = sum;
        }
    // twist / flip eigenvalues per pair (0,1), (0,2), (1,2), clamped
    double lp[3], lm[3];   // (lf + lt)/2 and (lf - lt)/2
    for (int k = 0; k < 3; ++k) {
        const int i = k == 2 ? 1 : 0, j = k == 0 ? 1 : 2;
        const double r = c / (sg[i] * sg[j]);
        const double lt = fmax(mu - r, 0.0), lf = fmax(mu + r, 0.0);
        lp[k] = 0.5 * (lf + lt);
        lm[k] = 0.5 * (lf - lt);
    }
    // d_m = V^T D[m]
    double d[12];
    for (int m = 0; m < 4; ++m)
        for (int s = 0; s < 3; ++s)
            d[3 * m + s] = D[3 * m] * V[s] + D[3 * m + 1] * V[3 + s] + D[3 * m + 2] * V[6 + s];
    for (int m = 0; m < 4; ++m)
        for (int n = m; n < 4; ++n) {
            const double* dm = d + 3 * m;
            const double* dn = d + 3 * n;
            double M[9];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) M[3 * r + s] = dm[r] * dn[s] * Ah[3 * r + s];
            for (int k = 0; k < 3; ++k) {
                const int i = k == 2 ? 1 : 0, j = k == 0 ? 1 : 2;
                M[4 * i] += lp[k] * dm[j] * dn[j];
                M[4 * j] += lp[k] * dm[i] * dn[i];
                M[3 * i + j] += lm[k] * dm[j] * dn[i];
                M[3 * j + i] += lm[k] * dm[i] * dn[j];
            }
            double T[9];   // U M
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 3; ++s) T[3 * a + s] = U[3 * a] * M[s] + U[3 * a + 1] * M[3 + s] + U[3 * a + 2] * M[6 + s];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double v = vol * (T[3 * a] * U[3 * b] + T[3 * a + 1] * U[3 * b + 1] + T[3 * a + 2] * U[3 * b + 2]);
                    out[(3 * m + a) * 12 + 3 * n + b] = v;
                    if (n != m) out[(3 * n + b) * 12 + 3 * m + a] = v;
                }
        }
}

// energy, gradient [nt][12] and (WANT_HESS) PSD Hessian [nt][144] per tet
template <bool WANT_HESS>
__global__ void __launch_bounds__(128)
k_nh_eval(ElasticView E, const double* __restrict__ x, double* __restrict__ tE,
          double* __restrict__ tG, double* __restrict__ tH, int32_t* __restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    double x4[12], X4[12], F[9], lnJ, psi;
    load_tet(E, x, t, x4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    const double vol = E.vol[t];
    if (!nh_energy(Dmi, vol, E.mu, E.lam, x4, X4, &psi, F, &lnJ)) {
        atomicMax(bad, 1);
        tE[t] = INFINITY;
        for (int q = 0; q < 12; ++q) tG[12 * t + q] = 0.0;
        if (WANT_HESS)
            for (int q = 0; q < 144; ++q) tH[144 * t + q] = 0.0;
        return;
    }
    tE[t] = psi;
    double Fi[9], G[9];
    inv3(F, Fi);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[3 * i + j] = Fi[3 * j + i];
    double D[12];   // D[m][j] = dF_ij / dx_{m,i}
    for (int j = 0; j < 3; ++j) {
        D[3 + j] = Dmi[j]; D[6 + j] = Dmi[3 + j]; D[9 + j] = Dmi[6 + j];
        D[j] = -(D[3 + j] + D[6 + j] + D[9 + j]);
    }
    double P[9];
    for (int i = 0; i < 9; ++i) P[i] = E.mu * (F[i] - G[i]) + E.lam * lnJ * G[i];
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += P[3 * i + j] * D[3 * m + j];
            tG[12 * t + 3 * m + i] = vol * s;
        }
    if (WANT_HESS) nh_hessian_blocks(F, lnJ, E.mu, E.lam, D, vol, tH + 144 * t);
}

// elastic energies at x + alpha_j p for j < na (<= 8), layout [na][nt]
__global__ void k_nh_energy_multi(ElasticView E, const double* __restrict__ x,
                                  const double* __restrict__ p, const double* __restrict__ alphas, int na,
                                  double* __restrict__ tE8) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    double x4[12], p4[12], X4[12], y4[12], F[9], lnJ, psi;
    load_tet(E, x, t, x4);
    load_tet(E, p, t, p4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    for (int j = 0; j < na; ++j) {
        const double a = alphas[j];
        for (int q = 0; q < 12; ++q) y4[q] = x4[q] + a * p4[q];
        tE8[(int64_t)j * E.nt + t] = nh_energy(Dmi, E.vol[t], E.mu, E.lam, y4, X4, &psi, F, &lnJ) ? psi : INFINITY;
    }
}

// G = M (x - xhat) + h^2 (sum_tets g + contact g); Dirichlet rows zero
__global__ void k_assemble_grad(int64_t nv, const double* __restrict__ x, const double* __restrict__ xhat,
                                const double* __restrict__ mass, const uint8_t* __restrict__ dir,
                                const int32_t* __restrict__ vt_off, const int32_t* __restrict__ vt_ent,
                                const double* __restrict__ tG, const void* __restrict__ cgrad, int cgrad_f32,
                                double h2, double* __restrict__ G) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    if (dir[v]) { G[3 * v] = 0.0; G[3 * v + 1] = 0.0; G[3 * v + 2] = 0.0; return; }
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int k = vt_off[v]; k < vt_off[v + 1]; ++k) {
        const int ent = vt_ent[k];
        const int64_t t = ent >> 2;
        const int a = ent & 3;
        e0 += tG[12 * t + 3 * a]; e1 += tG[12 * t + 3 * a + 1]; e2 += tG[12 * t + 3 * a + 2];
    }
    double c0, c1, c2;
    if (cgrad_f32) {
        const float* g = (const float*)cgrad;
        c0 = g[3 * v]; c1 = g[3 * v + 1]; c2 = g[3 * v + 2];
    } else {
        const double* g = (const double*)cgrad;
        c0 = g[3 * v]; c1 = g[3 * v + 1]; c2 = g[3 * v + 2];
    }
    const double m = mass[v];
    G[3 * v] = m * (x[3 * v] - xhat[3 * v]) + h2 * (e0 + c0);
    G[3 * v + 1] = m * (x[3 * v + 1] - xhat[3 * v + 1]) + h2 * (e1 + c1);
    G[3 * v + 2] = m * (x[3 * v + 2] - xhat[3 * v + 2]) + h2 * (e2 + c2);
}

// A = M + h^2 (sum_tets H + contact H) block by block; a block in a
// Dirichlet row or column is the identity on the diagonal and zero elsewhere
__global__ void k_assemble_bsr(int64_t nnzb, const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                               const int32_t* __restrict__ bt_off, const int32_t* __restrict__ bt_ent,
                               const double* __restrict__ tH, const int32_t* __restrict__ cmap,
                               const void* __restrict__ cvals, int cvals_f32,
                               const double* __restrict__ mass, const uint8_t* __restrict__ dir,
                               double h2, double* __restrict__ A) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnzb) return;
    const int i = brow[b], j = bcol[b];
    double* out = A + 9 * b;
    if (dir[i] || dir[j]) {
        for (int q = 0; q < 9; ++q) out[q] = (i == j && (q == 0 || q == 4 || q == 8)) ? 1.0 : 0.0;
        return;
    }
    double s[9];
    for (int q = 0; q < 9; ++q) s[q] = 0.0;
    for (int k = bt_off[b]; k < bt_off[b + 1]; ++k) {
        const int ent = bt_ent[k];
        const int64_t t = ent >> 4;
        const int ma = (ent >> 2) & 3, nb = ent & 3;
        const double* H = tH + 144 * t;
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) s[3 * p + q] += H[(3 * ma + p) * 12 + 3 * nb + q];
    }
    const int cb = cmap[b];
    if (cb >= 0) {
        if (cvals_f32) {
            const float* C = (const float*)cvals + 9 * (int64_t)cb;
            for (int q = 0; q < 9; ++q) s[q] += (double)C[q];
        } else {
            const double* C = (const double*)cvals + 9 * (int64_t)cb;
            for (int q = 0; q < 9; ++q) s[q] += C[q];
        }
    }
    for (int q = 0; q < 9; ++q) out[q] = h2 * s[q];
    if (i == j) { out[0] += mass[i]; out[4] += mass[i]; out[8] += mass[i]; }
}

// ------------------------------------------------------------------ PCG ---
__global__ void k_diag_inv(int64_t nv, const int32_t* __restrict__ diag_blk, const double* __restrict__ A,
                           double* __restrict__ Pinv) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    inv3(A + 9 * (int64_t)diag_blk[v], Pinv + 9 * v);
}

// y = A x, one thread per block row
__global__ void k_spmv(int64_t nv, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const double* B = A + 9 * (int64_t)k;
        const int64_t j = ci[k];
        const double x0 = x[3 * j], x1 = x[3 * j + 1], x2 = x[3 * j + 2];
        a0 += B[0] * x0 + B[1] * x1 + B[2] * x2;
        a1 += B[3] * x0 + B[4] * x1 + B[5] * x2;
        a2 += B[6] * x0 + B[7] * x1 + B[8] * x2;
    }
    y[3 * i] = a0; y[3 * i + 1] = a1; y[3 * i + 2] = a2;
}

__global__ void k_precond(int64_t nv, const double* __restrict__ Pinv, const double* __restrict__ r,
                          double* __restrict__ z) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const double* P = Pinv + 9 * i;
    const double r0 = r[3 * i], r1 = r[3 * i + 1], r2 = r[3 * i + 2];
    z[3 * i] = P[0] * r0 + P[1] * r1 + P[2] * r2;
    z[3 * i + 1] = P[3] * r0 + P[4] * r1 + P[5] * r2;
    z[3 * i + 2] = P[6] * r0 + P[7] * r1 + P[8] * r2;
}

// elementwise products into w (for a fixed-order dot product)
__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = a[i] * b[i];
}

// p = z + (rz_new / rz_old) p
__global__ void k_cg_dir(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                         double* __restrict__ p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double be = scal[2] / scal[0];
    p[i] = z[i] + be * p[i];
}

__global__ void k_copy_scal(double* __restrict__ scal, int dst, int src) { scal[dst] = scal[src]; }

// x += al p; r -= al Ap, unless p^T A p <= 0 (then flag scal[5] and keep x)
__global__ void k_cg_update_guarded(int64_t n, double* __restrict__ scal, double* __restrict__ x,
                                    double* __restrict__ r, const double* __restrict__ p,
                                    const double* __restrict__ Ap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!(scal[1] > 0.0)) {
        if (i == 0) scal[5] = 1.0;
        return;
    }
    if (i >= n) return;
    const double al = scal[0] / scal[1];
    x[i] += al * p[i];
    r[i] -= al * Ap[i];
}

// inertia terms 1/2 m |x + a_j p - xhat|^2 per vertex, layout [na][nv]
__global__ void k_inertia_multi(int64_t nv, const double* __restrict__ x, const double* __restrict__ p,
                                const double* __restrict__ xhat, const double* __restrict__ mass,
                                const double* __restrict__ alphas, int na, double* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double m = mass[v];
    for (int j = 0; j < na; ++j) {
        const double a = alphas[j];
        double e = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double d = (p ? x[3 * v + c] + a * p[3 * v + c] : x[3 * v + c]) - xhat[3 * v + c];
            e += 0.5 * m * d * d;
        }
        out[(int64_t)j * nv + v] = e;
    }
}

// E_j = Ein_j + h^2 (Ee_j + Ec_j)
__global__ void k_combine(int na, const double* __restrict__ ein, const double* __restrict__ ee,
                          const double* __restrict__ ec, double h2, double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= na) return;
    const double c = ec ? ec[j] : 0.0;
    out[j] = (isfinite(ee[j]) && isfinite(c)) ? ein[j] + h2 * (ee[j] + c) : INFINITY;
}

// ---------------------------------------------------------------- vectors ---
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, const double* __restrict__ p,
                       double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i] + a * p[i];
}
__global__ void k_xhat(int64_t nv, const double* __restrict__ x, const double* __restrict__ v, double h,
                       double g0, double g1, double g2, double* __restrict__ xhat) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const double g[3] = {g0, g1, g2};
    for (int c = 0; c < 3; ++c) xhat[3 * i + c] = x[3 * i + c] + h * v[3 * i + c] + h * h * g[c];
}
__global__ void k_dir_delta(int64_t nv, const uint8_t* __restrict__ dir, const double* __restrict__ x,
                            const double* __restrict__ xhat, double* __restrict__ dP) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int c = 0; c < 3; ++c) dP[3 * i + c] = dir[i] ? xhat[3 * i + c] - x[3 * i + c] : 0.0;
}
__global__ void k_set_dir(int64_t nv, const uint8_t* __restrict__ dir, const double* __restrict__ src,
                          double* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv || !dir[i]) return;
    for (int c = 0; c < 3; ++c) dst[3 * i + c] = src[3 * i + c];
}
__global__ void k_free_delta(int64_t nv, const uint8_t* __restrict__ dir, const double* __restrict__ P,
                             const double* __restrict__ xi, double* __restrict__ dP) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int c = 0; c < 3; ++c) dP[3 * i + c] = dir[i] ? 0.0 : P[3 * i + c] - xi[3 * i + c];
}
__global__ void k_zero_dir(int64_t nv, const uint8_t* __restrict__ dir, double* __restrict__ p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv || !dir[i]) return;
    p[3 * i] = 0.0; p[3 * i + 1] = 0.0; p[3 * i + 2] = 0.0;
}
__global__ void k_velocity(int64_t n, const double* __restrict__ x, const double* __restrict__ xt, double h,
                           double* __restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (x[i] - xt[i]) / h;
}
__global__ void k_neg(int64_t n, const double* __restrict__ a, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = -a[i];
}
}  // namespace

// ---------------------------------------------------------------------------
// host-side helpers used by the Newton driver in api.cu
// ---------------------------------------------------------------------------
static unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t nh_eval(Ctx& c, const double* x, bool want_hess, double* energy_dev, int32_t* bad) {
    NewtonState& N = *c.newton;
    ElasticView E{c.nt, N.tets.p, N.Dminv.p, N.vol.p, c.X.p, N.mu, N.lam};
    if (c.nt == 0) return cudaSuccess;
    if (want_hess)
        k_nh_eval<true><<<nblk(c.nt, 128), 128, 0, c.stream>>>(E, x, N.tE.p, N.tG.p, N.tH.p, bad);
    else
        k_nh_eval<false><<<nblk(c.nt, 128), 128, 0, c.stream>>>(E, x, N.tE.p, N.tG.p, N.tH.p, bad);
    GMCP_CUDA_TRY(cudaGetLastError());
    return reduce_sum(c, N.tE.p, c.nt, energy_dev);
}

cudaError_t nh_energy_multi(Ctx& c, const double* x, const double* p, const double* alphas_dev,
                            int na, double* energies_dev) {
    NewtonState& N = *c.newton;
    ElasticView E{c.nt, N.tets.p, N.Dminv.p, N.vol.p, c.X.p, N.mu, N.lam};
    if (c.nt == 0) return cudaMemsetAsync(energies_dev, 0, sizeof(double) * na, c.stream);
    k_nh_energy_multi<<<nblk(c.nt, 128), 128, 0, c.stream>>>(E, x, p, alphas_dev, na, N.tE8.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    for (int j = 0; j < na; ++j) GMCP_CUDA_TRY(reduce_sum(c, N.tE8.p + (int64_t)j * c.nt, c.nt, energies_dev + j));
    return cudaSuccess;
}

cudaError_t assemble_grad(Ctx& c, const double* x, const double* xhat, const void* cgrad, bool cgrad_f32,
                          double* G) {
    NewtonState& N = *c.newton;
    const double h2 = c.prm.h * c.prm.h;
    k_assemble_grad<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, x, xhat, N.mass.p, N.dir.p, N.vte_off.p,
                                                          N.vte.p, N.tG.p, cgrad, cgrad_f32 ? 1 : 0, h2, G);
    return cudaGetLastError();
}

cudaError_t assemble_bsr(Ctx& c) {
    NewtonState& N = *c.newton;
    const double h2 = c.prm.h * c.prm.h;
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    const void* cv = f32 ? (const void*)c.cb_val32.p : (const void*)c.cb_val64.p;
    k_assemble_bsr<<<nblk(N.nnzb, 256), 256, 0, c.stream>>>(N.nnzb, N.brow.p, N.bcol.p, N.bt_off.p, N.bt.p,
                                                           N.tH.p, N.cmap.p, cv, f32 ? 1 : 0, N.mass.p,
                                                           N.dir.p, h2, N.A.p);
    return cudaGetLastError();
}

// dot(a, b) -> out (device), fixed order
cudaError_t dot_dev(Ctx& c, const double* a, const double* b, int64_t n, double* out) {
    NewtonState& N = *c.newton;
    k_mul<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, b, N.w.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    return reduce_sum(c, N.w.p, n, out);
}

// Block-Jacobi PCG for A p = b (A = N.A on the pattern N.rp / N.ci), p = 0
// start; stops at ||r|| <= rel_tol ||b||, at p^T A p <= 0 or after max_it
// iterations.  One host readback per iteration.  Returns the iterations.
cudaError_t pcg_solve(Ctx& c, const double* b, double* xout, double rel_tol, int max_it, int* iters) {
    NewtonState& N = *c.newton;
    const int64_t n = 3 * c.nv;
    cudaStream_t s = c.stream;
    double* r = N.r.p; double* z = N.z.p; double* p = N.p.p; double* Ap = N.Ap.p;
    double* sc = N.scal.p;   // [0] rz  [1] pAp  [2] rz_new  [3] rr  [4] bb  [5] breakdown flag
    double* hb = c.h_scalars;
    *iters = 0;
    GMCP_CUDA_TRY(cudaMemsetAsync(xout, 0, sizeof(double) * n, s));
    GMCP_CUDA_TRY(cudaMemsetAsync(sc, 0, 8 * sizeof(double), s));
    GMCP_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    k_diag_inv<<<nblk(c.nv, 256), 256, 0, s>>>(c.nv, N.diag.p, N.A.p, N.Pinv.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(dot_dev(c, b, b, n, sc + 4));
    GMCP_CUDA_TRY(cudaMemcpyAsync(hb, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
    GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    const double bn = sqrt(hb[0]);
    if (!(bn > 0.0)) return cudaSuccess;
    k_precond<<<nblk(c.nv, 256), 256, 0, s>>>(c.nv, N.Pinv.p, r, z);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GMCP_CUDA_TRY(dot_dev(c, r, z, n, sc + 0));
    int it = 0;
    for (it = 0; it < max_it; ++it) {
        k_spmv<<<nblk(c.nv, 128), 128, 0, s>>>(c.nv, N.rp.p, N.ci.p, N.A.p, p, Ap);
        GMCP_CUDA_TRY(cudaGetLastError());
        GMCP_CUDA_TRY(dot_dev(c, p, Ap, n, sc + 1));
        k_cg_update_guarded<<<nblk(n, 256), 256, 0, s>>>(n, sc, xout, r, p, Ap);
        GMCP_CUDA_TRY(cudaGetLastError());
        GMCP_CUDA_TRY(dot_dev(c, r, r, n, sc + 3));
        GMCP_CUDA_TRY(cudaMemcpyAsync(hb, sc + 3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
        if (hb[2] != 0.0) break;                      // p^T A p <= 0: x unchanged
        if (sqrt(hb[0]) <= rel_tol * bn) { ++it; break; }
        k_precond<<<nblk(c.nv, 256), 256, 0, s>>>(c.nv, N.Pinv.p, r, z);
        GMCP_CUDA_TRY(cudaGetLastError());
        GMCP_CUDA_TRY(dot_dev(c, r, z, n, sc + 2));
        k_cg_dir<<<nblk(n, 256), 256, 0, s>>>(n, sc, z, p);
        k_copy_scal<<<1, 1, 0, s>>>(sc, 0, 2);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    *iters = it;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// setup: tet data, lumped mass and the global block pattern
// ---------------------------------------------------------------------------
static void h_inv3(const double* A, double* I) {
    const double d = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
    I[0] = (A[4] * A[8] - A[5] * A[7]) / d; I[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    I[2] = (A[1] * A[5] - A[2] * A[4]) / d; I[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    I[4] = (A[0] * A[8] - A[2] * A[6]) / d; I[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    I[6] = (A[3] * A[7] - A[4] * A[6]) / d; I[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    I[8] = (A[0] * A[4] - A[1] * A[3]) / d;
}

cudaError_t newton_setup(Ctx& c) {
    if (c.newton) return cudaSuccess;
    auto Np = std::make_unique<NewtonState>();
    NewtonState& N = *Np;
    const int64_t nv = c.nv, nt = c.nt;
    cudaStream_t s = c.stream;
    const ipc_params& q = c.prm;
    N.mu = q.youngs / (2.0 * (1.0 + q.poisson));
    N.lam = q.youngs * q.poisson / ((1.0 + q.poisson) * (1.0 - 2.0 * q.poisson));
    std::vector<double> Dminv(9 * (size_t)nt), vol(nt), mass(nv, 0.0);
    const int32_t* T = c.h_tets.data();
    const double* X = c.h_X.data();
    double vsum = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* Tt = T + 4 * t;
        double Dm[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) Dm[3 * r + k] = X[3 * Tt[k + 1] + r] - X[3 * Tt[0] + r];
        const double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                           Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
        vol[t] = fabs(det) / 6.0;
        vsum += vol[t];
        h_inv3(Dm, &Dminv[9 * t]);
        for (int a = 0; a < 4; ++a) mass[Tt[a]] += q.density * vol[t] / 4.0;
    }
    N.lbar = nt > 0 ? cbrt(vsum / (double)nt) : 0.0;
    // block pattern: diagonal, tet adjacency, contact pattern
    std::vector<int64_t> keys;
    keys.reserve((size_t)nv + 16 * (size_t)nt + c.h_cb_col.size());
    auto key = [nv](int64_t i, int64_t j) { return i * nv + j; };
    for (int64_t v = 0; v < nv; ++v) keys.push_back(key(v, v));
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) keys.push_back(key(T[4 * t + a], T[4 * t + b]));
    for (int64_t i = 0; i < nv; ++i)
        for (int k = c.h_cb_row[i]; k < c.h_cb_row[i + 1]; ++k) keys.push_back(key(i, c.h_cb_col[k]));
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    const int64_t nnzb = (int64_t)keys.size();
    if (nnzb >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    N.nnzb = nnzb;
    std::vector<int32_t> rp(nv + 1, 0), ci(nnzb), brow(nnzb), diag(nv);
    for (int64_t k = 0; k < nnzb; ++k) {
        brow[k] = (int32_t)(keys[k] / nv);
        ci[k] = (int32_t)(keys[k] % nv);
        rp[brow[k] + 1]++;
        if (brow[k] == ci[k]) diag[brow[k]] = (int32_t)k;
    }
    for (int64_t v = 0; v < nv; ++v) rp[v + 1] += rp[v];
    auto find = [&](int64_t i, int64_t j) -> int64_t {
        auto it = std::lower_bound(keys.begin() + rp[i], keys.begin() + rp[i + 1], key(i, j));
        return (it != keys.begin() + rp[i + 1] && *it == key(i, j)) ? (int64_t)(it - keys.begin()) : -1;
    };
    // per-block tet contributions in increasing (tet, a, b)
    std::vector<int32_t> bt_off(nnzb + 1, 0), bt(16 * (size_t)nt);
    std::vector<int64_t> tb(16 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int64_t k = find(T[4 * t + a], T[4 * t + b]);
                tb[16 * t + 4 * a + b] = k;
                bt_off[k + 1]++;
            }
    for (int64_t k = 0; k < nnzb; ++k) bt_off[k + 1] += bt_off[k];
    {
        std::vector<int32_t> cur(bt_off.begin(), bt_off.end() - 1);
        for (int64_t e = 0; e < 16 * nt; ++e) bt[cur[tb[e]]++] = (int32_t)e;
    }
    // vertex -> tet corner, increasing tet
    std::vector<int32_t> vte_off(nv + 1, 0), vte(4 * (size_t)nt);
    for (int64_t e = 0; e < 4 * nt; ++e) vte_off[T[e] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vte_off[v + 1] += vte_off[v];
    {
        std::vector<int32_t> cur(vte_off.begin(), vte_off.end() - 1);
        for (int64_t e = 0; e < 4 * nt; ++e) vte[cur[T[e]]++] = (int32_t)e;
    }
    // global block -> contact block
    std::vector<int32_t> cmap(nnzb, -1);
    for (int64_t i = 0; i < nv; ++i)
        for (int k = c.h_cb_row[i]; k < c.h_cb_row[i + 1]; ++k) cmap[find(i, c.h_cb_col[k])] = k;

    const size_t n3 = 3 * (size_t)nv;
    GMCP_CUDA_TRY(N.tets.upload(T, 4 * (size_t)nt, s));
    GMCP_CUDA_TRY(N.Dminv.upload(Dminv.data(), Dminv.size(), s));
    GMCP_CUDA_TRY(N.vol.upload(vol.data(), vol.size(), s));
    GMCP_CUDA_TRY(N.mass.upload(mass.data(), mass.size(), s));
    GMCP_CUDA_TRY(N.dir.upload(c.h_dir.data(), c.h_dir.size(), s));
    GMCP_CUDA_TRY(N.vte_off.upload(vte_off.data(), vte_off.size(), s));
    GMCP_CUDA_TRY(N.vte.upload(vte.data(), vte.size(), s));
    GMCP_CUDA_TRY(N.rp.upload(rp.data(), rp.size(), s));
    GMCP_CUDA_TRY(N.ci.upload(ci.data(), ci.size(), s));
    GMCP_CUDA_TRY(N.brow.upload(brow.data(), brow.size(), s));
    GMCP_CUDA_TRY(N.bcol.upload(ci.data(), ci.size(), s));
    GMCP_CUDA_TRY(N.diag.upload(diag.data(), diag.size(), s));
    GMCP_CUDA_TRY(N.bt_off.upload(bt_off.data(), bt_off.size(), s));
    GMCP_CUDA_TRY(N.bt.upload(bt.data(), bt.size(), s));
    GMCP_CUDA_TRY(N.cmap.upload(cmap.data(), cmap.size(), s));
    GMCP_CUDA_TRY(N.tE.ensure((size_t)nt + 1));
    GMCP_CUDA_TRY(N.tG.ensure(12 * (size_t)nt + 12));
    GMCP_CUDA_TRY(N.tH.ensure(144 * (size_t)nt + 144));
    GMCP_CUDA_TRY(N.tE8.ensure(8 * (size_t)nt + 8));
    GMCP_CUDA_TRY(N.A.ensure(9 * (size_t)nnzb));
    GMCP_CUDA_TRY(N.Pinv.ensure(9 * (size_t)nv));
    for (DBuf<double>* b : {&N.r, &N.z, &N.p, &N.Ap, &N.w, &N.xhat, &N.xt, &N.G, &N.dirn, &N.tmp, &N.P, &N.dP, &N.xi})
        GMCP_CUDA_TRY(b->ensure(n3));
    if (c.P.precision == IPC_PREC_MIXED) GMCP_CUDA_TRY(N.cgrad32.ensure(n3));
    else GMCP_CUDA_TRY(N.cgrad64.ensure(n3));
    GMCP_CUDA_TRY(N.xm.ensure(3 * (size_t)c.nmv + 3));
    GMCP_CUDA_TRY(N.dxm.ensure(3 * (size_t)c.nmv + 3));
    if (c.nmv > 0)
        GMCP_CUDA_TRY(cudaMemcpyAsync(N.xm.p, c.Y0.p, sizeof(double) * 3 * c.nmv, cudaMemcpyDeviceToDevice, s));
    GMCP_CUDA_TRY(N.ein8.ensure(8 * (size_t)nv));
    GMCP_CUDA_TRY(N.triE8.ensure(8 * (size_t)c.ns + 8));
    GMCP_CUDA_TRY(N.alphas.ensure(8));
    GMCP_CUDA_TRY(N.scal.ensure(64));
    GMCP_CUDA_TRY(N.bad.ensure(4));
    // host vectors must outlive the asynchronous copies
    GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    c.newton = std::move(Np);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// energies and the assembled system
// ---------------------------------------------------------------------------
// total incremental potential at x + alphas[j] p, j < na (<= 8), into
// out_dev[j]; the contact term is the frozen-linear potential of the samples
// active at x (requires the candidate lists of x)
cudaError_t energy_batch(Ctx& c, const double* x, const double* p, const double* alphas_dev, int na,
                         bool with_contact, double* out_dev) {
    NewtonState& N = *c.newton;
    double* sc = N.scal.p;   // [16..23] Ein  [24..31] Ee  [32..39] Ec
    GMCP_CUDA_TRY(nh_energy_multi(c, x, p, alphas_dev, na, sc + 24));
    k_inertia_multi<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, x, p, N.xhat.p, N.mass.p, alphas_dev, na, N.ein8.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    for (int j = 0; j < na; ++j) GMCP_CUDA_TRY(reduce_sum(c, N.ein8.p + (int64_t)j * c.nv, c.nv, sc + 16 + j));
    if (with_contact) GMCP_CUDA_TRY(contact_lagged(c, x, N.xm.p, p, alphas_dev, na, N.triE8.p, sc + 32));
    const double h2 = c.prm.h * c.prm.h;
    k_combine<<<1, 32, 0, c.stream>>>(na, sc + 16, sc + 24, with_contact ? sc + 32 : nullptr, h2, out_dev);
    return cudaGetLastError();
}

// E, gradient G (Dirichlet rows zero), optionally the matrix A, and |G|^2 at
// x; the broad phase runs at (x, current master).  Outputs: Ec_dev, Ee_dev
// (contact and elastic potentials), E_dev (total), gnorm2_dev, and the
// inverted-tet flag in N.bad.
cudaError_t assemble_system(Ctx& c, const double* x, bool want_hess, double* Ec_dev, double* Ee_dev,
                            double* E_dev, double* gnorm2_dev) {
    NewtonState& N = *c.newton;
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    GMCP_CUDA_TRY(cudaMemsetAsync(N.bad.p, 0, sizeof(int32_t), c.stream));
    {
        ProfScope ps(c.prof, c.stream, "elastic");
        GMCP_CUDA_TRY(nh_eval(c, x, want_hess, Ee_dev, N.bad.p));
    }
    GMCP_CUDA_TRY(run_candidates(c, x, N.xm.p));
    void* cg = f32 ? (void*)N.cgrad32.p : (void*)N.cgrad64.p;
    GMCP_CUDA_TRY(contact_eval(c, x, N.xm.p, Ec_dev, cg, want_hess, nullptr));
    {
        ProfScope ps(c.prof, c.stream, "assemble");
        GMCP_CUDA_TRY(assemble_grad(c, x, N.xhat.p, cg, f32, N.G.p));
        if (want_hess) GMCP_CUDA_TRY(assemble_bsr(c));
    }
    // total energy: inertia at x (slot 0 with alpha 0, p unused)
    double* sc = N.scal.p;
    const double zero = 0.0;
    GMCP_CUDA_TRY(cudaMemcpyAsync(N.alphas.p, &zero, sizeof(double), cudaMemcpyHostToDevice, c.stream));
    k_inertia_multi<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, x, nullptr, N.xhat.p, N.mass.p, N.alphas.p, 1, N.ein8.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(reduce_sum(c, N.ein8.p, c.nv, sc + 40));
    const double h2 = c.prm.h * c.prm.h;
    k_combine<<<1, 32, 0, c.stream>>>(1, sc + 40, Ee_dev, Ec_dev, h2, E_dev);
    GMCP_CUDA_TRY(cudaGetLastError());
    return dot_dev(c, N.G.p, N.G.p, 3 * c.nv, gnorm2_dev);
}

// --------------------------------------------------------------- vectors ---
cudaError_t vec_axpy(Ctx& c, int64_t n, double a, const double* x, const double* p, double* out) {
    k_axpy<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, x, p, out);
    return cudaGetLastError();
}
cudaError_t vec_xhat(Ctx& c, const double* x, const double* v, double* xhat) {
    const double* g = c.prm.gravity;
    k_xhat<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, x, v, c.prm.h, g[0], g[1], g[2], xhat);
    return cudaGetLastError();
}
cudaError_t vec_dir_delta(Ctx& c, const double* x, const double* xhat, double* dP) {
    k_dir_delta<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, c.newton->dir.p, x, xhat, dP);
    return cudaGetLastError();
}
cudaError_t vec_set_dir(Ctx& c, const double* src, double* dst) {
    k_set_dir<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, c.newton->dir.p, src, dst);
    return cudaGetLastError();
}
cudaError_t vec_free_delta(Ctx& c, const double* P, const double* xi, double* dP) {
    k_free_delta<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, c.newton->dir.p, P, xi, dP);
    return cudaGetLastError();
}
cudaError_t vec_zero_dir(Ctx& c, double* p) {
    k_zero_dir<<<nblk(c.nv, 256), 256, 0, c.stream>>>(c.nv, c.newton->dir.p, p);
    return cudaGetLastError();
}
cudaError_t vec_velocity(Ctx& c, const double* x, const double* xt, double* v) {
    const int64_t n = 3 * c.nv;
    k_velocity<<<nblk(n, 256), 256, 0, c.stream>>>(n, x, xt, c.prm.h, v);
    return cudaGetLastError();
}
cudaError_t vec_neg(Ctx& c, int64_t n, const double* a, double* out) {
    k_neg<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, out);
    return cudaGetLastError();
}

}  // namespace gmcp
