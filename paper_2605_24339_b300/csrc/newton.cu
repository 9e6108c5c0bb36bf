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
#include "dfloat.cuh"

namespace gmcp {
namespace {

__device__ __forceinline__ double det3(const double* A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
// (one FP64 division: the cofactors times 1/det; B300's FP64 divide is a
// long sequence on the slow pipe)
__device__ __forceinline__ void inv3(const double* A, double* I) {
    const double r = 1.0 / det3(A);
    I[0] = (A[4] * A[8] - A[5] * A[7]) * r; I[1] = (A[2] * A[7] - A[1] * A[8]) * r;
    I[2] = (A[1] * A[5] - A[2] * A[4]) * r; I[3] = (A[5] * A[6] - A[3] * A[8]) * r;
    I[4] = (A[0] * A[8] - A[2] * A[6]) * r; I[5] = (A[2] * A[3] - A[0] * A[5]) * r;
    I[6] = (A[3] * A[7] - A[4] * A[6]) * r; I[7] = (A[1] * A[6] - A[0] * A[7]) * r;
    I[8] = (A[0] * A[4] - A[1] * A[3]) * r;
}

// (J - 1) - ln J without cancellation, d = J - 1 and l = ln J = log1p(d):
// Taylor series for |d| < 1e-2 (truncation below 1e-17 relative), else the
// plain difference
__device__ __forceinline__ double d_minus_log1p(double d, double l) {
    if (fabs(d) < 1e-2)
        return d * d * (1.0 / 2 - d * (1.0 / 3 - d * (1.0 / 4 - d * (1.0 / 5 - d * (1.0 / 6 - d * (1.0 / 7 - d * (1.0 / 8 - d * (1.0 / 9))))))));
    return d - l;
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
// u = x - X, q = sum of principal 2x2 minors of H + det H and J - 1 = tr H + q
// (the energy and the inversion test below share it, so they decide J > 0
// alike)
__device__ __forceinline__ void nh_strain(const double* Dmi, const double* x4, const double* X4, double* H,
                                          double* q, double* jm1) {
    double u[12];
    for (int k = 0; k < 12; ++k) u[k] = x4[k] - X4[k];
    for (int i = 0; i < 3; ++i) {
        const double d1 = u[3 + i] - u[i], d2 = u[6 + i] - u[i], d3 = u[9 + i] - u[i];
        for (int j = 0; j < 3; ++j) H[3 * i + j] = d1 * Dmi[j] + d2 * Dmi[3 + j] + d3 * Dmi[6 + j];
    }
    const double trH = H[0] + H[4] + H[8];
    const double minors = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
    *q = minors + det3(H);
    *jm1 = trH + *q;
}

// F = I + H and the Neo-Hookean energy of the tet in the form
//   V [mu ((J-1) - ln J - q) + mu/2 |H|^2 + lambda/2 (ln J)^2],
//   J - 1 = tr H + q, q = sum of principal 2x2 minors of H + det H,
// (algebraically mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2, with the
// first-order terms cancelled exactly so the energy keeps its relative
// precision at small strain).  Returns false if J <= 0; else also J itself,
// formed as 1 + (J - 1).
__device__ __forceinline__ bool nh_energy(const double* Dmi, double vol, double mu, double lam,
                                          const double* x4, const double* X4, double* psi, double* F,
                                          double* lnJ, double* J) {
    double H[9], q, jm1;
    nh_strain(Dmi, x4, X4, H, &q, &jm1);
    for (int i = 0; i < 9; ++i) F[i] = H[i];
    F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
    if (!(jm1 > -1.0)) return false;
    double nH = 0.0;
    for (int i = 0; i < 9; ++i) nH += H[i] * H[i];
    *lnJ = log1p(jm1);
    *psi = vol * (mu * (d_minus_log1p(jm1, *lnJ) - q) + 0.5 * mu * nH + 0.5 * lam * (*lnJ) * (*lnJ));
    *J = 1.0 + jm1;
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
template <class R>
__device__ __forceinline__ void jacobi3(R* A, R* V) {
    const R tol2 = sizeof(R) == 4 ? R(1e-13) : R(1e-33);
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? R(1) : R(0);
#pragma unroll 1
    for (int sweep = 0; sweep < 32; ++sweep) {
        const R off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const R tot = off + R(0.5) * (A[0] * A[0] + A[4] * A[4] + A[8] * A[8]);
        if (off <= tol2 * tot || off == R(0)) break;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2;
            const R apq = A[3 * p + q];
            if (apq == R(0)) continue;
            const R theta = (A[3 * q + q] - A[3 * p + p]) / (R(2) * apq);
            const R t = (theta >= R(0) ? R(1) : R(-1)) / (fabs(theta) + sqrt(theta * theta + R(1)));
            const R c = R(1) / sqrt(t * t + R(1)), s = t * c;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const R arp = A[3 * r + p], arq = A[3 * r + q];
                A[3 * r + p] = c * arp - s * arq;
                A[3 * r + q] = s * arp + c * arq;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const R apr = A[3 * p + r], aqr = A[3 * q + r];
                A[3 * p + r] = c * apr - s * aqr;
                A[3 * q + r] = s * apr + c * aqr;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const R vrp = V[3 * r + p], vrq = V[3 * r + q];
                V[3 * r + p] = c * vrp - s * vrq;
                V[3 * r + q] = s * vrp + c * vrq;
            }
        }
    }
}

// the 10 distinct 3x3 blocks (m <= n) of a tet's 12x12 Hessian: block
// (m, n) is stored at kTetBlk[m] + n - m, row-major; (n, m) is its transpose
__constant__ int kTetBlk[4] = {0, 4, 7, 9};

// Each 3x3 block of the per-tet Hessian is stored with a stride of 48 bytes
// (12 FP32 or, rounded up, 10 FP64 entries; the tail unused), so that the
// assembly reads a block with 16-byte loads: [nt][10][kStride]
template <class T>
struct HBlk {
    static constexpr int kStride = sizeof(T) == 4 ? 12 : 10;
    static constexpr int kPerTet = 10 * kStride;
};
__device__ __forceinline__ void store_hblk(float* H, const float* h) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
        reinterpret_cast<float4*>(H)[c] = make_float4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
}
__device__ __forceinline__ void store_hblk(double* H, const double* h) {
#pragma unroll
    for (int c = 0; c < 5; ++c) reinterpret_cast<double2*>(H)[c] = make_double2(h[2 * c], h[2 * c + 1]);
}
__device__ __forceinline__ void load_hblk(const float* H, float* h) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(H));
    const float4 v = __ldg(reinterpret_cast<const float4*>(H) + 1);
    h[0] = u.x; h[1] = u.y; h[2] = u.z; h[3] = u.w;
    h[4] = v.x; h[5] = v.y; h[6] = v.z; h[7] = v.w;
    h[8] = __ldg(H + 8);
}
__device__ __forceinline__ void load_hblk(const double* H, double* h) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double2 u = __ldg(reinterpret_cast<const double2*>(H) + c);
        h[2 * c] = u.x; h[2 * c + 1] = u.y;
    }
    h[8] = __ldg(H + 8);
}

// PSD-projected Neo-Hookean Hessian of one tet, written as its 10 distinct
// 3x3 blocks in precision R.  dP/dF of an isotropic energy has a closed-form
// eigensystem in the singular values of F = U diag(s) V^T (Smith, de Goes,
// Kim 2019, "Analytic eigensystems for isotropic distortion energies"); for
// this energy, with c = mu - lambda ln J:
//   twist modes U (e_i e_j^T - e_j e_i^T) V^T / sqrt 2:  mu - c / (s_i s_j)
//   flip modes  U (e_i e_j^T + e_j e_i^T) V^T / sqrt 2:  mu + c / (s_i s_j)
//   scaling modes U diag(e) V^T, e the eigenvectors of the 3x3
//     A_ii = mu + (c + lambda) / s_i^2, A_ij = lambda / (s_i s_j).
// Clamping the eigenvalues at zero gives the same (unique) projection as a
// 9x9 eigen-decomposition.  With D[m] the rows of dF/dx and d_m = V^T D[m],
// block (m, n) = V_tet U M_mn U^T, M_mn = sum_k max(l_k, 0) (E_k d_m)(E_k d_n)^T.
template <class R, class In = double>
__device__ void nh_hessian_blocks(const In* Fd, In lnJd, In mud, In lamd, const In* Dmi, In vold,
                                  R* out /* [10][HBlk<R>::kStride] */) {
    R F[9], D[12];   // D[m][j] = dF_ij / dx_{m,i}: rows 1..3 of D are Dm^-1, row 0 minus their sum
    for (int i = 0; i < 9; ++i) F[i] = (R)Fd[i];
    for (int j = 0; j < 3; ++j) {
        D[3 + j] = (R)Dmi[j]; D[6 + j] = (R)Dmi[3 + j]; D[9 + j] = (R)Dmi[6 + j];
        D[j] = -(D[3 + j] + D[6 + j] + D[9 + j]);
    }
    const R mu = (R)mud, lam = (R)lamd, vol = (R)vold;
    // SVD from the eigen-decomposition of F^T F
    R S[9], V[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    jacobi3(S, V);
    const R detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                   V[2] * (V[3] * V[7] - V[4] * V[6]);
    if (detV < R(0)) { V[2] = -V[2]; V[5] = -V[5]; V[8] = -V[8]; }
    R B[9];   // F V, columns b_k
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) B[3 * i + k] = F[3 * i] * V[k] + F[3 * i + 1] * V[3 + k] + F[3 * i + 2] * V[6 + k];
    R U[9], sg[3];
    {
        const R n0 = sqrt(B[0] * B[0] + B[3] * B[3] + B[6] * B[6]);
        const R u0[3] = {B[0] / n0, B[3] / n0, B[6] / n0};
        const R pr = u0[0] * B[1] + u0[1] * B[4] + u0[2] * B[7];
        const R w1[3] = {B[1] - pr * u0[0], B[4] - pr * u0[1], B[7] - pr * u0[2]};
        const R n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
        R u1[3];
        if (n1 > R(1e-30) * n0) {
            u1[0] = w1[0] / n1; u1[1] = w1[1] / n1; u1[2] = w1[2] / n1;
        } else {   // any unit vector orthogonal to u0
            const R ax = fabs(u0[0]), ay = fabs(u0[1]), az = fabs(u0[2]);
            R e[3] = {R(0), R(0), R(0)};
            e[(ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2)] = R(1);
            const R d = e[0] * u0[0] + e[1] * u0[1] + e[2] * u0[2];
            const R w[3] = {e[0] - d * u0[0], e[1] - d * u0[1], e[2] - d * u0[2]};
            const R nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            u1[0] = w[0] / nw; u1[1] = w[1] / nw; u1[2] = w[2] / nw;
        }
        const R u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
        sg[0] = n0;
        sg[1] = u1[0] * B[1] + u1[1] * B[4] + u1[2] * B[7];
        sg[2] = u2[0] * B[2] + u2[1] * B[5] + u2[2] * B[8];
        for (int i = 0; i < 3; ++i) { U[3 * i] = u0[i]; U[3 * i + 1] = u1[i]; U[3 * i + 2] = u2[i]; }
    }
    const R c = (R)(mud - lamd * lnJd);
    // scaling block and its projection
    R A[9], W[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = (i == j) ? mu + (c + lam) / (sg[i] * sg[i]) : lam / (sg[i] * sg[j]);
    // its projection is A itself where A is certainly positive definite
    // (Sylvester's criterion, the determinant above 1e-6 (FP32) / 1e-12
    // (FP64) of the cube of its largest entry, far above rounding);
    // otherwise from its eigen-decomposition
    R Ah[9];
    const R m2 = A[0] * A[4] - A[1] * A[3];
    const R d3 = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    R amax = R(0);
    for (int q = 0; q < 9; ++q) amax = fmax(amax, fabs(A[q]));
    const R tol_pd = sizeof(R) == 4 ? R(1e-6) : R(1e-12);
    if (A[0] > R(0) && m2 > R(0) && d3 > tol_pd * amax * amax * amax) {
        for (int q = 0; q < 9; ++q) Ah[q] = A[q];
    } else {
        jacobi3(A, W);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                R sum = R(0);
                for (int k = 0; k < 3; ++k) {
                    const R l = A[4 * k];
                    if (l > R(0)) sum += W[3 * i + k] * l * W[3 * j + k];
                }
                Ah[3 * i + j] = sum;
            }
    }
    // twist / flip eigenvalues per pair (0,1), (0,2), (1,2), clamped
    R lp[3], lm[3];   // (lf + lt)/2 and (lf - lt)/2
    for (int k = 0; k < 3; ++k) {
        const int i = k == 2 ? 1 : 0, j = k == 0 ? 1 : 2;
        const R r = c / (sg[i] * sg[j]);
        const R lt = fmax(mu - r, R(0)), lf = fmax(mu + r, R(0));
        lp[k] = R(0.5) * (lf + lt);
        lm[k] = R(0.5) * (lf - lt);
    }
    // d_m = V^T D[m]
    R d[12];
    for (int m = 0; m < 4; ++m)
        for (int s = 0; s < 3; ++s)
            d[3 * m + s] = D[3 * m] * V[s] + D[3 * m + 1] * V[3 + s] + D[3 * m + 2] * V[6 + s];
    int blk = 0;
    for (int m = 0; m < 4; ++m)
        for (int n = m; n < 4; ++n, ++blk) {
            const R* dm = d + 3 * m;
            const R* dn = d + 3 * n;
            R M[9];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) M[3 * r + s] = dm[r] * dn[s] * Ah[3 * r + s];
            for (int k = 0; k < 3; ++k) {
                const int i = k == 2 ? 1 : 0, j = k == 0 ? 1 : 2;
                M[4 * i] += lp[k] * dm[j] * dn[j];
                M[4 * j] += lp[k] * dm[i] * dn[i];
                M[3 * i + j] += lm[k] * dm[j] * dn[i];
                M[3 * j + i] += lm[k] * dm[i] * dn[j];
            }
            R T[9];   // U M
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 3; ++s) T[3 * a + s] = U[3 * a] * M[s] + U[3 * a + 1] * M[3 + s] + U[3 * a + 2] * M[6 + s];
            R hb[HBlk<R>::kStride];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    hb[3 * a + b] = vol * (T[3 * a] * U[3 * b] + T[3 * a + 1] * U[3 * b + 1] + T[3 * a + 2] * U[3 * b + 2]);
            for (int q = 9; q < HBlk<R>::kStride; ++q) hb[q] = R(0);   // whole sectors are written
            store_hblk(out + HBlk<R>::kStride * blk, hb);
        }
}

// energy, gradient [nt][12] and (WANT_HESS) PSD Hessian [nt][10][stride] (10 blocks,
// precision TH) per tet
template <bool WANT_HESS, class TH>
__global__ void __launch_bounds__(128)
k_nh_eval(ElasticView E, const double* __restrict__ x, double* __restrict__ tE,
          double* __restrict__ tG, TH* __restrict__ tH, int32_t* __restrict__ bad,
          const int32_t* __restrict__ tet_env) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    double x4[12], X4[12], F[9], lnJ, J, psi;
    load_tet(E, x, t, x4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    const double vol = E.vol[t];
    if (!nh_energy(Dmi, vol, E.mu, E.lam, x4, X4, &psi, F, &lnJ, &J)) {
        atomicMax(bad + (tet_env ? tet_env[t] : 0), 1);
        tE[t] = INFINITY;
        for (int q = 0; q < 12; ++q) tG[12 * t + q] = 0.0;
        if (WANT_HESS)
            for (int q = 0; q < HBlk<TH>::kPerTet; ++q) tH[HBlk<TH>::kPerTet * t + q] = TH(0);
        return;
    }
    tE[t] = psi;
    // first Piola stress times the volume, V (mu (F - F^-T) + lambda ln J F^-T),
    // with F^-T = C / J (C the cofactor matrix of F):
    //   V P = (mu V) F + ((lambda ln J - mu) V / J) C
    double C[9];
    C[0] = F[4] * F[8] - F[5] * F[7]; C[1] = F[5] * F[6] - F[3] * F[8]; C[2] = F[3] * F[7] - F[4] * F[6];
    C[3] = F[2] * F[7] - F[1] * F[8]; C[4] = F[0] * F[8] - F[2] * F[6]; C[5] = F[1] * F[6] - F[0] * F[7];
    C[6] = F[1] * F[5] - F[2] * F[4]; C[7] = F[2] * F[3] - F[0] * F[5]; C[8] = F[0] * F[4] - F[1] * F[3];
    const double mv = E.mu * vol, cv = (E.lam * lnJ - E.mu) * vol / J;
    double P[9];
    for (int i = 0; i < 9; ++i) P[i] = mv * F[i] + cv * C[i];
    // gradient rows: vertex m >= 1 gets P (Dm^-1 row m-1), vertex 0 minus their sum
    for (int i = 0; i < 3; ++i) {
        double s0 = 0.0;
        for (int m = 1; m < 4; ++m) {
            const double* d = Dmi + 3 * (m - 1);
            const double sm = P[3 * i] * d[0] + P[3 * i + 1] * d[1] + P[3 * i + 2] * d[2];
            tG[12 * t + 3 * m + i] = sm;
            s0 += sm;
        }
        tG[12 * t + i] = -s0;
    }
    if (WANT_HESS) nh_hessian_blocks<TH>(F, lnJ, E.mu, E.lam, Dmi, vol, tH + HBlk<TH>::kPerTet * t);
}

// elastic energies at x + alpha_j p for j < na (<= 8), layout [na][nt]
// (alphas of tet t's environment: alphas[astride * env + j])
// (base: subtract each tet's energy at x, base[t], to give the change)
__global__ void k_nh_energy_multi(ElasticView E, const double* __restrict__ x,
                                  const double* __restrict__ p, const double* __restrict__ alphas_env, int astride,
                                  const int32_t* __restrict__ tet_env, int na, double* __restrict__ tE8,
                                  const double* __restrict__ base) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    const double* alphas = alphas_env + (int64_t)astride * tet_env[t];
    double x4[12], p4[12], X4[12], y4[12], F[9], lnJ, J, psi;
    load_tet(E, x, t, x4);
    load_tet(E, p, t, p4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    for (int j = 0; j < na; ++j) {
        const double a = alphas[j];
        for (int q = 0; q < 12; ++q) y4[q] = x4[q] + a * p4[q];
        const bool ok = nh_energy(Dmi, E.vol[t], E.mu, E.lam, y4, X4, &psi, F, &lnJ, &J);
        tE8[(int64_t)j * E.nt + t] = ok ? (base ? psi - base[t] : psi) : INFINITY;
    }
}

// inversion test at x + alpha_j p for j < na (<= 8): 0 where the tet keeps
// J > 0, +inf where not (the energy's own test, without the energy), layout
// [na][nt]
__global__ void k_nh_feasible(ElasticView E, const double* __restrict__ x, const double* __restrict__ p,
                              const double* __restrict__ alphas_env, int astride,
                              const int32_t* __restrict__ tet_env, int na, double* __restrict__ tE8) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    const double* alphas = alphas_env + (int64_t)astride * tet_env[t];
    double x4[12], p4[12], X4[12], y4[12], H[9], q, jm1;
    load_tet(E, x, t, x4);
    load_tet(E, p, t, p4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    for (int j = 0; j < na; ++j) {
        const double a = alphas[j];
        for (int k = 0; k < 12; ++k) y4[k] = x4[k] + a * p4[k];
        nh_strain(Dmi, y4, X4, H, &q, &jm1);
        tE8[(int64_t)j * E.nt + t] = jm1 > -1.0 ? 0.0 : INFINITY;
    }
}

// ---------------------------------------------- mixed path: double-float ---
// The same elastic terms (the same formulas and branch points as the FP64
// kernels above) in double-float arithmetic (about 48 bits, on the FP32
// pipe): the displacement u = x - X and a direction p enter split into
// pairs once per vertex (k_split_pairs), Dm^-1 and the volumes once at setup.
struct ElasticViewDF {
    int64_t nt;
    const int32_t* tets;
    const float2* Dmi;   // [nt][9]
    const float2* vol;   // [nt]
    dfl mu, lam;
    dfl c13, c15, c23;   // 1/3, 1/5, 2/3 as pairs (series coefficients)
};

// u = x - X (or p alone when X is null) split into pairs, [nv][4] hi and lo
__global__ void k_split_pairs(int64_t nv, const double* __restrict__ x, const double* __restrict__ X,
                              float4* __restrict__ hi, float4* __restrict__ lo) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    dfl d[3];
    for (int c = 0; c < 3; ++c) d[c] = df_from_double(X ? x[3 * v + c] - X[3 * v + c] : x[3 * v + c]);
    hi[v] = make_float4(d[0].hi, d[1].hi, d[2].hi, 0.f);
    lo[v] = make_float4(d[0].lo, d[1].lo, d[2].lo, 0.f);
}

__device__ __forceinline__ dfl ld_pair(const float2* p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}
__device__ __forceinline__ void load_tet_pairs(const ElasticViewDF& E, const float4* hi, const float4* lo, int64_t t,
                                               dfl* u4) {
    for (int a = 0; a < 4; ++a) {
        const int64_t v = E.tets[4 * t + a];
        const float4 h = __ldg(hi + v), l = __ldg(lo + v);
        u4[3 * a] = {h.x, l.x}; u4[3 * a + 1] = {h.y, l.y}; u4[3 * a + 2] = {h.z, l.z};
    }
}

// nh_strain in pairs
__device__ __forceinline__ void nh_strain_df(const dfl* Dmi, const dfl* u, dfl* H, dfl* q, dfl* jm1) {
    for (int i = 0; i < 3; ++i) {
        const dfl d1 = df_sub(u[3 + i], u[i]), d2 = df_sub(u[6 + i], u[i]), d3 = df_sub(u[9 + i], u[i]);
        for (int j = 0; j < 3; ++j) H[3 * i + j] = df_fma(d3, Dmi[6 + j], df_fma(d2, Dmi[3 + j], df_mul(d1, Dmi[j])));
    }
    const dfl trH = df_add(df_add(H[0], H[4]), H[8]);
    const dfl c00 = df_mms(H[4], H[8], H[5], H[7]);
    const dfl minors = df_add(df_add(df_mms(H[0], H[4], H[1], H[3]), df_mms(H[0], H[8], H[2], H[6])), c00);
    const dfl det = df_add(df_sub(df_mul(H[0], c00), df_mul(H[1], df_mms(H[3], H[8], H[5], H[6]))),
                           df_mul(H[2], df_mms(H[3], H[7], H[4], H[6])));
    *q = df_add(minors, det);
    *jm1 = df_add(trH, *q);
}

// ln J = log1p(d) and (J - 1) - ln J for d = J - 1: for |d| < 1e-2 by
// series, ln(1 + d) = 2 atanh(s) = 2 (s + s^3/3 + ... + s^9/9) with
// s = d / (2 + d) (|s| < 5e-3, truncation below 4e-19 relative), and
// d - ln(1 + d) = d^2 (1/2 - d/3 + d^2/4 - ... + d^7/9) (as in the FP64
// kernels); otherwise in FP64 from the pair's value (no cancellation there)
__device__ __forceinline__ void nh_log_df(const ElasticViewDF& E, dfl d, dfl* lnJ, dfl* dml) {
    if (fabsf(d.hi) < 1e-2f) {
        const dfl s = df_div(d, df_add(df_make(2.f), d));
        const dfl t = df_mul(s, s);
        const float in = 0.4f + t.hi * (2.f / 7.f + t.hi * (2.f / 9.f));
        const dfl c1 = df_add(E.c23, df_mulf(t, in));
        *lnJ = df_mul(s, df_add(df_make(2.f), df_mul(t, c1)));
        const float tail = 1.f / 6.f - d.hi * (1.f / 7.f - d.hi * (1.f / 8.f - d.hi * (1.f / 9.f)));
        const dfl s5 = df_sub(E.c15, df_mulf(d, tail));
        const dfl s4 = df_sub(df_make(0.25f), df_mul(d, s5));
        const dfl s3 = df_sub(E.c13, df_mul(d, s4));
        const dfl s2 = df_sub(df_make(0.5f), df_mul(d, s3));
        *dml = df_mul(df_mul(d, d), s2);
    } else {
        const double jd = df_to_double(d);
        const double l = log1p(jd);
        *lnJ = df_from_double(l);
        *dml = df_from_double(jd - l);
    }
}

// nh_energy in pairs: false if J <= 0
__device__ __forceinline__ bool nh_energy_df(const ElasticViewDF& E, const dfl* Dmi, dfl vol, const dfl* u,
                                             dfl* psi, dfl* H, dfl* lnJ, dfl* jm1) {
    dfl q;
    nh_strain_df(Dmi, u, H, &q, jm1);
    if (!df_gt(*jm1, -1.f)) return false;
    dfl nH = df_mul(H[0], H[0]);
    for (int i = 1; i < 9; ++i) nH = df_fma(H[i], H[i], nH);
    dfl dml;
    nh_log_df(E, *jm1, lnJ, &dml);
    const dfl a = df_mul(E.mu, df_sub(dml, q));
    const dfl b = df_mul(E.mu, nH);
    const dfl l2 = df_mul(E.lam, df_mul(*lnJ, *lnJ));
    const dfl half = df_add(b, l2);
    *psi = df_mul(vol, df_add(a, {0.5f * half.hi, 0.5f * half.lo}));
    return true;
}

// k_nh_eval of the mixed path: energy (FP64 from the pair), gradient as
// pairs [nt][12], FP32 Hessian blocks from the pairs' high parts
template <bool WANT_HESS>
__global__ void __launch_bounds__(128)
k_nh_eval_df(ElasticViewDF E, const float4* __restrict__ uh, const float4* __restrict__ ul,
             double* __restrict__ tE, float2* __restrict__ tG, float* __restrict__ tH, int32_t* __restrict__ bad,
             const int32_t* __restrict__ tet_env) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    dfl u[12], Dmi[9], H[9], psi, lnJ, jm1;
    load_tet_pairs(E, uh, ul, t, u);
    for (int k = 0; k < 9; ++k) Dmi[k] = ld_pair(E.Dmi + 9 * t + k);
    const dfl vol = ld_pair(E.vol + t);
    if (!nh_energy_df(E, Dmi, vol, u, &psi, H, &lnJ, &jm1)) {
        atomicMax(bad + (tet_env ? tet_env[t] : 0), 1);
        tE[t] = INFINITY;
        for (int k = 0; k < 12; ++k) tG[12 * t + k] = make_float2(0.f, 0.f);
        if (WANT_HESS)
            for (int k = 0; k < HBlk<float>::kPerTet; ++k) tH[HBlk<float>::kPerTet * t + k] = 0.f;
        return;
    }
    tE[t] = df_to_double(psi);
    dfl F[9];
    for (int k = 0; k < 9; ++k) F[k] = H[k];
    F[0] = df_add(F[0], df_make(1.f)); F[4] = df_add(F[4], df_make(1.f)); F[8] = df_add(F[8], df_make(1.f));
    // V P = (mu V) F + ((lambda ln J - mu) V / J) C, C the cofactors of F
    dfl C[9];
    C[0] = df_mms(F[4], F[8], F[5], F[7]); C[1] = df_mms(F[5], F[6], F[3], F[8]); C[2] = df_mms(F[3], F[7], F[4], F[6]);
    C[3] = df_mms(F[2], F[7], F[1], F[8]); C[4] = df_mms(F[0], F[8], F[2], F[6]); C[5] = df_mms(F[1], F[6], F[0], F[7]);
    C[6] = df_mms(F[1], F[5], F[2], F[4]); C[7] = df_mms(F[2], F[3], F[0], F[5]); C[8] = df_mms(F[0], F[4], F[1], F[3]);
    const dfl J = df_add(df_make(1.f), jm1);
    const dfl mv = df_mul(E.mu, vol);
    const dfl cv = df_div(df_mul(df_sub(df_mul(E.lam, lnJ), E.mu), vol), J);
    dfl P[9];
    for (int k = 0; k < 9; ++k) P[k] = df_add(df_mul(mv, F[k]), df_mul(cv, C[k]));
    for (int i = 0; i < 3; ++i) {
        dfl s0 = df_make(0.f);
        for (int m = 1; m < 4; ++m) {
            const dfl* d = Dmi + 3 * (m - 1);
            const dfl sm = df_fma(P[3 * i + 2], d[2], df_fma(P[3 * i + 1], d[1], df_mul(P[3 * i], d[0])));
            tG[12 * t + 3 * m + i] = make_float2(sm.hi, sm.lo);
            s0 = df_add(s0, sm);
        }
        tG[12 * t + i] = make_float2(-s0.hi, -s0.lo);
    }
    if (WANT_HESS) {
        float Ff[9], Df[9];
        for (int k = 0; k < 9; ++k) { Ff[k] = F[k].hi; Df[k] = Dmi[k].hi; }
        nh_hessian_blocks<float, float>(Ff, lnJ.hi, E.mu.hi, E.lam.hi, Df, vol.hi, tH + HBlk<float>::kPerTet * t);
    }
}

// k_nh_energy_multi of the mixed path (changes from base: FP64 energies of
// the last evaluation at x)
__global__ void __launch_bounds__(128)
k_nh_energy_multi_df(ElasticViewDF E, const float4* __restrict__ uh, const float4* __restrict__ ul,
                     const float4* __restrict__ ph, const float4* __restrict__ pl,
                     const double* __restrict__ alphas_env, int astride, const int32_t* __restrict__ tet_env,
                     int na, double* __restrict__ tE8, const double* __restrict__ base) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    const double* alphas = alphas_env + (int64_t)astride * tet_env[t];
    dfl u[12], p[12], Dmi[9], y[12], H[9], psi, lnJ, jm1;
    load_tet_pairs(E, uh, ul, t, u);
    load_tet_pairs(E, ph, pl, t, p);
    for (int k = 0; k < 9; ++k) Dmi[k] = ld_pair(E.Dmi + 9 * t + k);
    const dfl vol = ld_pair(E.vol + t);
    for (int j = 0; j < na; ++j) {
        const dfl a = df_from_double(alphas[j]);
        for (int k = 0; k < 12; ++k) y[k] = df_fma(a, p[k], u[k]);
        double out = INFINITY;
        if (nh_energy_df(E, Dmi, vol, y, &psi, H, &lnJ, &jm1))
            out = base ? ((double)psi.hi - base[t]) + (double)psi.lo : df_to_double(psi);
        tE8[(int64_t)j * E.nt + t] = out;
    }
}

// k_nh_feasible of the mixed path
__global__ void __launch_bounds__(128)
k_nh_feasible_df(ElasticViewDF E, const float4* __restrict__ uh, const float4* __restrict__ ul,
                 const float4* __restrict__ ph, const float4* __restrict__ pl,
                 const double* __restrict__ alphas_env, int astride, const int32_t* __restrict__ tet_env, int na,
                 double* __restrict__ tE8) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    const double* alphas = alphas_env + (int64_t)astride * tet_env[t];
    dfl u[12], p[12], Dmi[9], y[12], H[9], q, jm1;
    load_tet_pairs(E, uh, ul, t, u);
    load_tet_pairs(E, ph, pl, t, p);
    for (int k = 0; k < 9; ++k) Dmi[k] = ld_pair(E.Dmi + 9 * t + k);
    for (int j = 0; j < na; ++j) {
        const dfl a = df_from_double(alphas[j]);
        for (int k = 0; k < 12; ++k) y[k] = df_fma(a, p[k], u[k]);
        nh_strain_df(Dmi, y, H, &q, &jm1);
        tE8[(int64_t)j * E.nt + t] = df_gt(jm1, -1.f) ? 0.0 : INFINITY;
    }
}

// The Hessian blocks alone, for a Newton iteration that goes on after the
// convergence test (the energy and gradient at x were evaluated without
// them): F and ln J from the same code as the evaluation, so the blocks are
// bitwise those k_nh_eval(_df) would have written; inverted tets get zero
// blocks (the evaluation flagged them).
__global__ void __launch_bounds__(128)
k_nh_hess_df(ElasticViewDF E, const float4* __restrict__ uh, const float4* __restrict__ ul,
             float* __restrict__ tH) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    dfl u[12], Dmi[9], H[9], q, jm1, lnJ, dml;
    load_tet_pairs(E, uh, ul, t, u);
    for (int k = 0; k < 9; ++k) Dmi[k] = ld_pair(E.Dmi + 9 * t + k);
    nh_strain_df(Dmi, u, H, &q, &jm1);
    if (!df_gt(jm1, -1.f)) {
        for (int k = 0; k < HBlk<float>::kPerTet; ++k) tH[HBlk<float>::kPerTet * t + k] = 0.f;
        return;
    }
    nh_log_df(E, jm1, &lnJ, &dml);
    float Ff[9], Df[9];
    for (int k = 0; k < 9; ++k) {
        Ff[k] = k % 4 == 0 ? df_add(H[k], df_make(1.f)).hi : H[k].hi;   // as k_nh_eval_df forms F
        Df[k] = Dmi[k].hi;
    }
    nh_hessian_blocks<float, float>(Ff, lnJ.hi, E.mu.hi, E.lam.hi, Df, ld_pair(E.vol + t).hi,
                                    tH + HBlk<float>::kPerTet * t);
}
__global__ void __launch_bounds__(128)
k_nh_hess64(ElasticView E, const double* __restrict__ x, double* __restrict__ tH) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E.nt) return;
    double x4[12], X4[12], F[9], lnJ, J, psi;
    load_tet(E, x, t, x4);
    load_tet(E, E.X, t, X4);
    const double* Dmi = E.Dminv + 9 * t;
    const double vol = E.vol[t];
    if (!nh_energy(Dmi, vol, E.mu, E.lam, x4, X4, &psi, F, &lnJ, &J)) {
        for (int k = 0; k < HBlk<double>::kPerTet; ++k) tH[HBlk<double>::kPerTet * t + k] = 0.0;
        return;
    }
    nh_hessian_blocks<double>(F, lnJ, E.mu, E.lam, Dmi, vol, tH + HBlk<double>::kPerTet * t);
}

// G = M (x - xhat) + h^2 (sum_tets g + contact g); Dirichlet rows zero
__global__ void k_assemble_grad(int64_t nv, const double* __restrict__ x, const double* __restrict__ xhat,
                                const double* __restrict__ mass, const uint8_t* __restrict__ dir,
                                const int32_t* __restrict__ vt_off, const int32_t* __restrict__ vt_ent,
                                const double* __restrict__ tG, int tg_pairs, const void* __restrict__ cgrad,
                                int cgrad_f32, const double* __restrict__ fext, double h2, double* __restrict__ G) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    if (dir[v]) { G[3 * v] = 0.0; G[3 * v + 1] = 0.0; G[3 * v + 2] = 0.0; return; }
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    if (tg_pairs) {   // per-tet gradients as FP32 pairs (mixed path): summed as pairs
        const float2* g = reinterpret_cast<const float2*>(tG);
        dfl s0 = df_make(0.f), s1 = df_make(0.f), s2 = df_make(0.f);
        for (int k = vt_off[v]; k < vt_off[v + 1]; ++k) {
            const int ent = vt_ent[k];
            const int64_t t = ent >> 2;
            const int a = ent & 3;
            s0 = df_add(s0, ld_pair(g + 12 * t + 3 * a));
            s1 = df_add(s1, ld_pair(g + 12 * t + 3 * a + 1));
            s2 = df_add(s2, ld_pair(g + 12 * t + 3 * a + 2));
        }
        e0 = df_to_double(s0); e1 = df_to_double(s1); e2 = df_to_double(s2);
    } else {
        for (int k = vt_off[v]; k < vt_off[v + 1]; ++k) {
            const int ent = vt_ent[k];
            const int64_t t = ent >> 2;
            const int a = ent & 3;
            e0 += tG[12 * t + 3 * a]; e1 += tG[12 * t + 3 * a + 1]; e2 += tG[12 * t + 3 * a + 2];
        }
    }
    double c0, c1, c2;
    if (cgrad_f32) {
        const float* g = (const float*)cgrad;
        c0 = g[3 * v]; c1 = g[3 * v + 1]; c2 = g[3 * v + 2];
    } else {
        const double* g = (const double*)cgrad;
        c0 = g[3 * v]; c1 = g[3 * v + 1]; c2 = g[3 * v + 2];
    }
    if (fext) {   // external forces: -h^2 f
        c0 -= fext[3 * v]; c1 -= fext[3 * v + 1]; c2 -= fext[3 * v + 2];
    }
    const double m = mass[v];
    G[3 * v] = m * (x[3 * v] - xhat[3 * v]) + h2 * (e0 + c0);
    G[3 * v + 1] = m * (x[3 * v + 1] - xhat[3 * v + 1]) + h2 * (e1 + c1);
    G[3 * v + 2] = m * (x[3 * v + 2] - xhat[3 * v + 2]) + h2 * (e2 + c2);
}

// Sliced-ELL storage of the matrix: rows are taken 32 at a time (a slice),
// each slice holds as many groups as its longest row has blocks, and group g
// holds the k-th blocks of its 32 rows (lane = row mod 32) in 288 entries.
// Entries 0..7 of a block sit in 16-byte vectors of VW = 16 / sizeof(TA)
// entries, vector c of all 32 lanes side by side; entry 8 follows for all
// lanes.  A warp thus reads a group with two (FP32) or four (FP64) coalesced
// 16-byte loads and one 4- or 8-byte load per thread.
template <class TA>
__host__ __device__ __forceinline__ int64_t sell_idx(int64_t g, int lane, int q) {
    constexpr int VW = 16 / (int)sizeof(TA);
    return q < 8 ? 288 * g + 32 * VW * (q / VW) + VW * lane + q % VW : 288 * g + 256 + lane;
}

// A = M + h^2 (sum_tets H + contact H) block by block in precision TA; a
// block in a Dirichlet row or column is the identity on the diagonal and zero
// elsewhere.  Only the blocks (i, j >= i) are stored (A is symmetric).  One
// thread per stored block, in storage order, so every store is coalesced;
// padding blocks are zero.
template <class TH, class TC, class TA>
__global__ void k_assemble_sell(int64_t nv, int64_t ngroups, const int32_t* __restrict__ goff,
                                const int32_t* __restrict__ gslice, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ llen, const int32_t* __restrict__ bcol,
                                const int32_t* __restrict__ bt_off,
                                const int32_t* __restrict__ bt_ent, const TH* __restrict__ tH,
                                const int32_t* __restrict__ cmap, const TC* __restrict__ cvals,
                                const double* __restrict__ xvals,
                                const double* __restrict__ mass, const uint8_t* __restrict__ dir, double h2,
                                TA* __restrict__ A) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = t >> 5;
    if (g >= ngroups) return;
    const int lane = (int)(t & 31);
    const int sl = gslice[g];
    const int k = (int)(g - goff[sl]);
    const int64_t i = 32 * (int64_t)sl + lane;
    const int ll = i < nv ? llen[i] : 0;
    const int len = i < nv ? rp[i + 1] - rp[i] - ll : 0;
    if (k >= len) {
        for (int q = 0; q < 9; ++q) A[sell_idx<TA>(g, lane, q)] = TA(0);
        return;
    }
    const int64_t b = rp[i] + ll + k;   // the k-th stored (j >= i) block of row i
    const int64_t j = bcol[b];
    if (dir[i] || dir[j]) {
        for (int q = 0; q < 9; ++q)
            A[sell_idx<TA>(g, lane, q)] = (i == j && (q == 0 || q == 4 || q == 8)) ? TA(1) : TA(0);
        return;
    }
    TA s[9];
    for (int q = 0; q < 9; ++q) s[q] = TA(0);
    for (int e = bt_off[b]; e < bt_off[b + 1]; ++e) {
        const int ent = bt_ent[e];
        const int64_t tt = ent >> 4;
        const int ma = (ent >> 2) & 3, nb = ent & 3;
        constexpr int HS = HBlk<TH>::kStride;
        TH h[9];
        if (ma <= nb) {
            load_hblk(tH + HBlk<TH>::kPerTet * tt + HS * (kTetBlk[ma] + nb - ma), h);
            for (int q = 0; q < 9; ++q) s[q] += (TA)h[q];
        } else {
            load_hblk(tH + HBlk<TH>::kPerTet * tt + HS * (kTetBlk[nb] + ma - nb), h);
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) s[3 * p + q] += (TA)h[3 * q + p];
        }
    }
    const int cb = cmap[b];
    if (cb >= 0) {
        const TC* C = cvals + 9 * (int64_t)cb;
        for (int q = 0; q < 9; ++q) s[q] += (TA)C[q];
    }
    if (xvals) {   // joint step: the blocks with master vertices
        const double* X9 = xvals + 9 * b;
        for (int q = 0; q < 9; ++q) s[q] += (TA)X9[q];
    }
    const TA h2a = (TA)h2;
    for (int q = 0; q < 9; ++q) s[q] *= h2a;
    if (i == j) {
        const TA m = (TA)mass[i];
        s[0] += m; s[4] += m; s[8] += m;
    }
    for (int q = 0; q < 9; ++q) A[sell_idx<TA>(g, lane, q)] = s[q];
}

// ------------------------------------------------- joint step: master entries ---
// The master rows and blocks come as an unordered list (row, col, 9 values;
// col -1 = a gradient row) from the sample kernels.  They are counted and
// placed by destination row (integer atomics), each row's entries sorted by
// (col, value bits) and every run of equal col summed in that order, so the
// sums do not depend on the order the list was written in.
__global__ void k_ml_count(const int32_t* __restrict__ ij, const unsigned long long* __restrict__ count,
                           int64_t cap, int64_t nsys, int32_t* __restrict__ cnt, int32_t* __restrict__ err) {
    const int64_t n = min((int64_t)*count, cap);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ij[2 * e];
        if (r < 0 || r >= nsys) { atomicExch(err, 2); continue; }
        atomicAdd(&cnt[r], 1);
    }
}
__global__ void k_ml_fill(const int32_t* __restrict__ ij, const unsigned long long* __restrict__ count, int64_t cap,
                          int64_t nsys, const int32_t* __restrict__ off, int32_t* __restrict__ cur,
                          int32_t* __restrict__ perm) {
    const int64_t n = min((int64_t)*count, cap);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ij[2 * e];
        if (r < 0 || r >= nsys) continue;
        perm[off[r] + atomicAdd(&cur[r], 1)] = (int32_t)e;
    }
}
__device__ __forceinline__ bool ml_less(const int32_t* ij, const double* blk, int32_t a, int32_t b) {
    const int32_t ca = ij[2 * (int64_t)a + 1], cb = ij[2 * (int64_t)b + 1];
    if (ca != cb) return ca < cb;
    for (int q = 0; q < 9; ++q) {
        const unsigned long long ua = (unsigned long long)__double_as_longlong(blk[9 * (int64_t)a + q]);
        const unsigned long long ub = (unsigned long long)__double_as_longlong(blk[9 * (int64_t)b + q]);
        if (ua != ub) return ua < ub;
    }
    return false;
}
// one thread per system row: sort, then sum the runs; rows (col -1) go to
// cgrad, blocks (col >= row) to xvals at their pattern position (the stored
// half; the entries (j, i) of a master-master pair are the transposes)
template <class TG>
__global__ void k_ml_reduce(int64_t nsys, const int32_t* __restrict__ off, int32_t* __restrict__ perm,
                            const int32_t* __restrict__ ij, const double* __restrict__ blk,
                            const int32_t* __restrict__ rp, const int32_t* __restrict__ llen,
                            const int32_t* __restrict__ ci, double* __restrict__ xvals, TG* __restrict__ cgrad,
                            int64_t row_base, int32_t* __restrict__ err) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nsys) return;
    const int32_t b0 = off[r], b1 = off[r + 1];
    for (int32_t k = b0 + 1; k < b1; ++k) {   // insertion sort (short rows)
        const int32_t v = perm[k];
        int32_t m = k - 1;
        while (m >= b0 && ml_less(ij, blk, v, perm[m])) { perm[m + 1] = perm[m]; --m; }
        perm[m + 1] = v;
    }
    for (int32_t k = b0; k < b1;) {
        const int32_t col = ij[2 * (int64_t)perm[k] + 1];
        double sum[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        int32_t k2 = k;
        for (; k2 < b1 && ij[2 * (int64_t)perm[k2] + 1] == col; ++k2) {
            const double* B = blk + 9 * (int64_t)perm[k2];
            for (int q = 0; q < 9; ++q) sum[q] += B[q];
        }
        k = k2;
        if (col < 0) {
            if (r >= row_base)
                for (int q = 0; q < 3; ++q) cgrad[3 * (r - row_base) + q] = (TG)sum[q];
        } else if (xvals && col >= r) {
            int32_t lo = rp[r] + llen[r], hi = rp[r + 1] - 1, at = -1;
            while (lo <= hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (ci[mid] == col) { at = mid; break; }
                if (ci[mid] < col) lo = mid + 1; else hi = mid - 1;
            }
            if (at < 0) { atomicExch(err, 1); continue; }
            for (int q = 0; q < 9; ++q) xvals[9 * (int64_t)at + q] = sum[q];
        }
    }
}

// ------------------------------------------------------------------ PCG ---
// Fused block-Jacobi PCG: three kernels per iteration, one thread per block
// row in each; each dot product is finished by the last block to arrive,
// which sums the per-block partials in block order (deterministic) and forms
// the iteration's scalars once (alpha in the SpMV kernel, beta in the update
// kernel), so no thread divides.  Vectors r, z, Ap ([nv][3]), the search
// direction p ([nv][4], the fourth entry unused, so a neighbour's three
// entries are one aligned load) and the block inverse are of type V (FP64,
// or FP32 in the mixed path).  Dot products are formed per thread and per
// warp in V and summed across warps and blocks in FP64 (the B300 FP64 pipe
// runs at 1/64 of FP32, so FP64 per element would dominate the mixed path).
// The solution is FP64 in the FP64 path and an unevaluated pair of floats
// (hi + lo, compensated summation) in the mixed path.  Solver scalars (FP64):
enum : int {
    kRz = 0,         // r . z of the current iteration
    kPAp = 1, kAl = 2, kBe = 3, kRr = 4, kBb = 5,
    kBreak = 6,      // p^T A p <= 0 seen
    kDone = 7,       // converged
    kIters = 8,      // iterations taken (valid once kBreak or kDone is set)
    kThr = 9,        // rel_tol |b|
    kIt = 10,        // index of the current iteration (advanced by k_pcg_update)
    kCtlI = 11,      // two int32: stop (break or done), iteration index
    kCtlF = 12       // two float: alpha, beta (FP32 copies)
};
// The control words repeat the stop flags, the iteration index and alpha,
// beta in int32 / FP32, so that the per-iteration kernels test and read them
// without FP64 instructions (each costs a full warp issue on the B300's
// narrow FP64 pipe).
constexpr int kEnvScal = 16;   // doubles of per-environment scalars
__device__ __forceinline__ int* pcg_ictl(double* scal) { return reinterpret_cast<int*>(scal + kCtlI); }
__device__ __forceinline__ float* pcg_fctl(double* scal) { return reinterpret_cast<float*>(scal + kCtlF); }
template <class V>
__device__ __forceinline__ V pcg_scalar(double* scal, int k /* kAl or kBe */) {
    if constexpr (sizeof(V) == 4) return pcg_fctl(scal)[k == kAl ? 0 : 1];
    else return scal[k];
}
constexpr int kPcgThreads = 256;

// Programmatic dependent launch: the PCG kernels are launched so that the
// next one may start while the previous one drains (its last block forms
// the iteration's scalars).  Each kernel waits for its predecessor's memory
// before reading anything the predecessor writes, and lets its successor
// launch as soon as it has passed that point.  Launched without the
// attribute, both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// whether the SpMV forms the search direction itself (FP32; see k_pcg_spmv)
template <class V>
struct PcgDir {
    static constexpr bool kFused = sizeof(V) == 4;
    static constexpr int kZs = kFused ? 4 : 3;   // row stride of z (4: gathered by the SpMV)
};

// block sums of v0 and v1 (NV = 1 or 2): a shuffle tree in R within each
// warp, then the eight warp sums in FP64 (fixed order); valid in warp 0
template <int NV, class R>
__device__ __forceinline__ void block_sums256(R v0, R v1, double (*sh)[kPcgThreads / 32], double* b0, double* b1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        if (NV > 1) v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = (double)v0;
        if (NV > 1) sh[1][threadIdx.x >> 5] = (double)v1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < kPcgThreads / 32;
        double r0 = in ? sh[0][threadIdx.x] : 0.0;
        double r1 = (NV > 1 && in) ? sh[1][threadIdx.x] : 0.0;
#pragma unroll
        for (int o = kPcgThreads / 64; o > 0; o >>= 1) {
            r0 += __shfl_xor_sync(0xffffffffu, r0, o);
            if (NV > 1) r1 += __shfl_xor_sync(0xffffffffu, r1, o);
        }
        *b0 = r0;
        *b1 = r1;
    }
}

// Each block contributes NV values (v0, v1) to its environment's sums;
// returns true in the environment's last block to arrive, where thread 0
// then holds the environment's fixed-order totals in *t0, *t1.  The blocks
// of one environment are consecutive (first block b_first, nb of them) and
// count at *counter; part is [2][gridDim].
template <int NV, class R>
__device__ bool last_block_sums(R v0, R v1, double* part, unsigned* counter, int b_first, int nb, double* t0,
                                double* t1) {
    __shared__ double sh[2][kPcgThreads / 32];
    __shared__ bool am_last;
    double b0 = 0.0, b1 = 0.0;
    block_sums256<NV, R>(v0, v1, sh, &b0, &b1);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b0;
        if (NV > 1) part[gridDim.x + blockIdx.x] = b1;
        __threadfence();
        am_last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    const volatile double* vp = part;
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < nb; k += kPcgThreads) {
        s0 += vp[b_first + k];
        if (NV > 1) s1 += vp[gridDim.x + b_first + k];
    }
    __syncthreads();   // the first pass's readers of sh are done
    block_sums256<NV, double>(s0, s1, sh, t0, t1);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

template <class V>
__device__ __forceinline__ void mul33(const V* P, V r0, V r1, V r2, V* z) {
    z[0] = P[0] * r0 + P[1] * r1 + P[2] * r2;
    z[1] = P[3] * r0 + P[4] * r1 + P[5] * r2;
    z[2] = P[6] * r0 + P[7] * r1 + P[8] * r2;
}

// the three used entries of p[i] (stride 4): one 16-byte load in FP32
__device__ __forceinline__ void load_p(const float* p, int64_t i, float& a, float& b, float& c) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    a = v.x; b = v.y; c = v.z;
}
__device__ __forceinline__ void load_p(const double* p, int64_t i, double& a, double& b, double& c) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p + 4 * i));
    a = v.x; b = v.y; c = __ldg(p + 4 * i + 2);
}

// the nine entries of the stored block (g, lane)
__device__ __forceinline__ void load_blk(const float* A, int64_t g, int lane, float* b) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(A + sell_idx<float>(g, lane, 0)));
    const float4 v = __ldg(reinterpret_cast<const float4*>(A + sell_idx<float>(g, lane, 4)));
    b[0] = u.x; b[1] = u.y; b[2] = u.z; b[3] = u.w;
    b[4] = v.x; b[5] = v.y; b[6] = v.z; b[7] = v.w;
    b[8] = __ldg(A + sell_idx<float>(g, lane, 8));
}
__device__ __forceinline__ void load_blk(const double* A, int64_t g, int lane, double* b) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double2 u = __ldg(reinterpret_cast<const double2*>(A + sell_idx<double>(g, lane, 2 * c)));
        b[2 * c] = u.x; b[2 * c + 1] = u.y;
    }
    b[8] = __ldg(A + sell_idx<double>(g, lane, 8));
}

// inverse of each diagonal block (inverted in FP64, stored as V); the
// diagonal is the first stored block of its row
template <class TA, class V>
__global__ void k_diag_inv(int64_t nv, const int32_t* __restrict__ goff, const TA* __restrict__ A,
                           const int32_t* __restrict__ vprow, V* __restrict__ Pinv) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double D[9], I[9];
    const int64_t g = goff[v >> 5];
    for (int q = 0; q < 9; ++q) D[q] = (double)A[sell_idx<TA>(g, (int)(v & 31), q)];
    inv3(D, I);
    const int64_t r = vprow[v];
    for (int q = 0; q < 9; ++q) Pinv[9 * r + q] = (V)I[q];
}

// x = 0, r = b, z = P^-1 b; p = z (FP64), or, where the SpMV forms the
// direction, p (first of the pair) = 0 and beta = 0 so that it forms p = z;
// b.b and r.z
// Launch geometry of the per-row kernels: block b covers rows [B.y, B.z) of
// environment B.x (B = blk[b]; B.w its environment's first block), so every
// dot product is a per-environment sum whose blocks start at the
// environment's first row.  Vertex-row kernels (init, SpMV): 256 vertex
// rows a block; padded-row kernels (update, direction): 512 padded rows.
template <class V>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_init(const int4* __restrict__ blk, const int32_t* __restrict__ env_nblk, const int32_t* __restrict__ vprow,
           const V* __restrict__ Pinv, const double* __restrict__ bvec, double* __restrict__ x,
           V* __restrict__ xh, V* __restrict__ xl, V* __restrict__ r, V* __restrict__ z, V* __restrict__ p, double* part,
           unsigned* counters, double* escal, double rel_tol) {
    const int4 B = blk[blockIdx.x];
    double* scal = escal + kEnvScal * B.x;
    const int64_t iv = (int64_t)B.y + threadIdx.x;   // vertex row
    V bb = V(0), rz = V(0);
    if (iv < B.z) {
        const int64_t i = vprow[iv];                  // padded row
        const V b0 = (V)bvec[3 * iv], b1 = (V)bvec[3 * iv + 1], b2 = (V)bvec[3 * iv + 2];
        V zz[3];
        mul33(Pinv + 9 * i, b0, b1, b2, zz);
        const V bv[3] = {b0, b1, b2};
        for (int q = 0; q < 3; ++q) {
            if (sizeof(V) == 8) {
                x[3 * iv + q] = 0.0;
            } else {
                xh[3 * i + q] = V(0);
                xl[3 * i + q] = V(0);
            }
            r[3 * i + q] = bv[q];
            z[PcgDir<V>::kZs * i + q] = zz[q];
            p[4 * i + q] = PcgDir<V>::kFused ? V(0) : zz[q];
            bb += bv[q] * bv[q];
            rz += bv[q] * zz[q];
        }
        if (PcgDir<V>::kZs == 4) z[4 * i + 3] = V(0);
        p[4 * i + 3] = V(0);
    }
    double tb, tr;
    if (last_block_sums<2, V>(bb, rz, part, counters + B.x, B.w, env_nblk[B.x], &tb, &tr) && threadIdx.x == 0) {
        scal[kBb] = tb;
        scal[kRz] = tr;
        scal[kThr] = rel_tol * sqrt(tb);
        scal[kBreak] = 0.0;
        scal[kDone] = tb > 0.0 ? 0.0 : 1.0;
        scal[kIters] = 0.0;
        scal[kIt] = 0.0;
        scal[kBe] = 0.0;   // a fused first SpMV forms p = z + 0 * p (p zero)
        pcg_ictl(scal)[0] = tb > 0.0 ? 0 : 1;
        pcg_ictl(scal)[1] = 0;
        pcg_fctl(scal)[1] = 0.f;
    }
}

// In FP32 the search direction is kept as a pair of buffers [2][nvp][4]:
// iteration it reads p_old = pair[it mod 2] and writes p_new = pair[(it + 1)
// mod 2].  p_new = z + beta p_old is formed by the SpMV itself, for its own
// row (stored) and for every neighbour it multiplies (recomputed from z and
// p_old, bitwise the same value), so no separate direction pass is needed:
// the extra neighbour reads hit L2 and cost less than a pass over p and z.
// In FP64 the recomputation would load the FP64 pipe (the B300's is 1/64
// of FP32), so there p is one buffer, updated by k_pcg_dir.
template <class V>
__device__ __forceinline__ void dir_row(const V* p_old, const V* z, int64_t j, V be, V& a, V& b, V& c) {
    V p0, p1, p2;
    load_p(p_old, j, p0, p1, p2);
    if constexpr (PcgDir<V>::kFused) {
        V z0, z1, z2;
        load_p(z, j, z0, z1, z2);
        a = fmaf(be, p0, z0); b = fmaf(be, p1, z1); c = fmaf(be, p2, z2);
    } else {
        a = p0; b = p1; c = p2;
    }
}

// Ap = A p_new and p_new.Ap; one thread per block row, over the row's blocks
// in column order (the transposed blocks j < i, then the stored ones), sums
// in TA.  The last block sets alpha = r.z / p.Ap (or
// the breakdown flag).
template <class TA, class V>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_spmv(const int4* __restrict__ blk, const int32_t* __restrict__ env_nblk, const int32_t* __restrict__ vprow,
           int64_t nvp, const int32_t* __restrict__ rp, const int32_t* __restrict__ goff,
           const int32_t* __restrict__ sci, const int32_t* __restrict__ llen, const int32_t* __restrict__ lgoff,
           const int32_t* __restrict__ lcol, const int32_t* __restrict__ lmir, const TA* __restrict__ A,
           V* __restrict__ ppair, const V* __restrict__ z, V* __restrict__ Ap, double* part, unsigned* counters,
           double* escal) {
    pdl_wait();
    pdl_trigger();
    const int4 B = blk[blockIdx.x];
    double* scal = escal + kEnvScal * B.x;
    if (pcg_ictl(scal)[0] != 0) return;
    const int it = pcg_ictl(scal)[1];
    constexpr bool kFused = PcgDir<V>::kFused;
    const V be = pcg_scalar<V>(scal, kBe);
    const V* p_old = kFused ? ppair + 4 * nvp * (it & 1) : ppair;
    V* p_new = ppair + 4 * nvp * ((it + 1) & 1);
    const int64_t i = (int64_t)B.y + threadIdx.x;   // vertex row (the matrix storage's row)
    V pap = V(0);
    if (i < B.z) {
        const int64_t ir = vprow[i];                  // its padded row (the vectors' row)
        const int64_t g0 = goff[i >> 5];
        const int lane = (int)(i & 31);
        const int ll = llen[i];
        const int len = rp[i + 1] - rp[i] - ll;
        const int32_t* cj = sci + 32 * g0 + lane;
        TA a0 = TA(0), a1 = TA(0), a2 = TA(0);
        // the blocks j < i first (column order): transposes of block (j, i)
        // in row j's storage, gathered (they were streamed by row j's slice
        // and are read from L2); the same pipeline as below
        if (ll > 0) {
            const int64_t lg0 = lgoff[i >> 5];
            const int32_t* lc = lcol + 32 * lg0 + lane;
            const int32_t* lm = lmir + 32 * lg0 + lane;
            TA bn[9];
            V qn0, qn1, qn2;
            int32_t m2 = 0;
            int64_t j2 = 0;
            {
                const int32_t m = __ldg(lm);
                load_blk(A, m >> 5, m & 31, bn);
                dir_row(p_old, z, __ldg(lc), be, qn0, qn1, qn2);
            }
            if (ll > 1) { j2 = __ldg(lc + 32); m2 = __ldg(lm + 32); }
            for (int k = 0; k < ll; ++k) {
                TA b[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) b[q] = bn[q];
                const TA p0 = (TA)qn0, p1 = (TA)qn1, p2 = (TA)qn2;
                if (k + 1 < ll) {
                    load_blk(A, m2 >> 5, m2 & 31, bn);
                    dir_row(p_old, z, j2, be, qn0, qn1, qn2);
                    if (k + 2 < ll) { j2 = __ldg(lc + 32 * (k + 2)); m2 = __ldg(lm + 32 * (k + 2)); }
                }
                a0 += b[0] * p0 + b[3] * p1 + b[6] * p2;
                a1 += b[1] * p0 + b[4] * p1 + b[7] * p2;
                a2 += b[2] * p0 + b[5] * p1 + b[8] * p2;
            }
        }
        // the stored blocks j >= i: software pipeline, the column two blocks
        // ahead, the block and the neighbour's direction one block ahead are
        // in flight while a block is multiplied
        TA bn[9];
        V qn0 = V(0), qn1 = V(0), qn2 = V(0);
        int64_t j2 = 0;
        if (len > 0) {
            load_blk(A, g0, lane, bn);
            dir_row(p_old, z, __ldg(cj), be, qn0, qn1, qn2);
        }
        if (len > 1) j2 = __ldg(cj + 32);
        for (int k = 0; k < len; ++k) {
            TA b[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) b[q] = bn[q];
            const TA p0 = (TA)qn0, p1 = (TA)qn1, p2 = (TA)qn2;
            if (k + 1 < len) {
                load_blk(A, g0 + k + 1, lane, bn);
                dir_row(p_old, z, j2, be, qn0, qn1, qn2);
                if (k + 2 < len) j2 = __ldg(cj + 32 * (k + 2));
            }
            a0 += b[0] * p0 + b[1] * p1 + b[2] * p2;
            a1 += b[3] * p0 + b[4] * p1 + b[5] * p2;
            a2 += b[6] * p0 + b[7] * p1 + b[8] * p2;
        }
        const V y0 = (V)a0, y1 = (V)a1, y2 = (V)a2;
        Ap[3 * ir] = y0;
        Ap[3 * ir + 1] = y1;
        Ap[3 * ir + 2] = y2;
        V q0, q1, q2;
        dir_row(p_old, z, ir, be, q0, q1, q2);
        if constexpr (kFused) reinterpret_cast<float4*>(p_new)[ir] = make_float4(q0, q1, q2, 0.f);
        pap = q0 * y0 + q1 * y1 + q2 * y2;
    }
    double t, unused;
    if (last_block_sums<1, V>(pap, V(0), part, counters + B.x, B.w, env_nblk[B.x], &t, &unused) &&
        threadIdx.x == 0) {
        scal[kPAp] = t;
        if (t > 0.0) {
            scal[kAl] = scal[kRz] / t;
            pcg_fctl(scal)[0] = (float)scal[kAl];
        } else {
            scal[kBreak] = 1.0;
            scal[kIters] = (double)it;
            pcg_ictl(scal)[0] = 1;
        }
    }
}

// rows handled by one thread of the update kernel: two, so that a thread's
// rows of every vector are whole 8-byte (FP32) or 16-byte (FP64) vectors
// (the vectors are padded to a multiple of four rows)
template <class V>
struct PcgRows {
    static constexpr int R = 2;
};

// n consecutive values of V: 16-byte vectors when n * sizeof(V) is a
// multiple of 16 (the address then 16-byte aligned), else 8-byte ones
template <class V, int N>
__device__ __forceinline__ void ldv(const V* __restrict__ src, V* dst) {
    if constexpr (sizeof(V) == 4 && (N * 4) % 16 != 0) {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const float2 u = __ldg(reinterpret_cast<const float2*>(src) + c);
            dst[2 * c] = u.x; dst[2 * c + 1] = u.y;
        }
    } else if constexpr (sizeof(V) == 4) {
#pragma unroll
        for (int c = 0; c < N / 4; ++c) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(src) + c);
            dst[4 * c] = u.x; dst[4 * c + 1] = u.y; dst[4 * c + 2] = u.z; dst[4 * c + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const double2 u = __ldg(reinterpret_cast<const double2*>(src) + c);
            dst[2 * c] = u.x; dst[2 * c + 1] = u.y;
        }
    }
}
template <class V, int N>
__device__ __forceinline__ void ldv_rw(const V* src, V* dst) {   // for buffers the kernel also writes
    if constexpr (sizeof(V) == 4 && (N * 4) % 16 != 0) {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const float2 u = reinterpret_cast<const float2*>(src)[c];
            dst[2 * c] = u.x; dst[2 * c + 1] = u.y;
        }
    } else if constexpr (sizeof(V) == 4) {
#pragma unroll
        for (int c = 0; c < N / 4; ++c) {
            const float4 u = reinterpret_cast<const float4*>(src)[c];
            dst[4 * c] = u.x; dst[4 * c + 1] = u.y; dst[4 * c + 2] = u.z; dst[4 * c + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const double2 u = reinterpret_cast<const double2*>(src)[c];
            dst[2 * c] = u.x; dst[2 * c + 1] = u.y;
        }
    }
}
template <class V, int N>
__device__ __forceinline__ void stv(V* dst, const V* src) {
    if constexpr (sizeof(V) == 4 && (N * 4) % 16 != 0) {
#pragma unroll
        for (int c = 0; c < N / 2; ++c)
            reinterpret_cast<float2*>(dst)[c] = make_float2(src[2 * c], src[2 * c + 1]);
    } else if constexpr (sizeof(V) == 4) {
#pragma unroll
        for (int c = 0; c < N / 4; ++c)
            reinterpret_cast<float4*>(dst)[c] = make_float4(src[4 * c], src[4 * c + 1], src[4 * c + 2], src[4 * c + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < N / 2; ++c)
            reinterpret_cast<double2*>(dst)[c] = make_double2(src[2 * c], src[2 * c + 1]);
    }
}

// hi + lo += v (Knuth's two-sum; |lo| stays below half an ulp of hi)
__device__ __forceinline__ void add_pair(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bv = s - hi;
    const float e = (hi - (s - bv)) + (v - bv);
    hi = s;
    lo += e;
}

// x += al p, r -= al Ap, z = P^-1 r (z: [nvp][4], the fourth entry zero),
// then r.r (convergence) and r.z; the last block sets beta = r.z_new / r.z
// and advances the iteration index.
// PcgRows<V>::R rows per thread over the padded rows nvp; x is FP64 (rows
// below nv) when V is FP64, else the float pair (xh, xl).
template <class V>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_update(const int4* __restrict__ blk, const int32_t* __restrict__ env_nblk, const int32_t* __restrict__ prow_v,
             int64_t nvp, const V* __restrict__ Pinv, double* __restrict__ x, V* __restrict__ xh,
             V* __restrict__ xl, V* __restrict__ r, V* __restrict__ z, const V* __restrict__ ppair,
             const V* __restrict__ Ap, double* part, unsigned* counters, double* escal) {
    constexpr int R = PcgRows<V>::R;
    pdl_wait();
    pdl_trigger();
    const int4 B = blk[blockIdx.x];
    double* scal = escal + kEnvScal * B.x;
    if (pcg_ictl(scal)[0] != 0) return;
    const int it = pcg_ictl(scal)[1];
    const V* p = PcgDir<V>::kFused ? ppair + 4 * nvp * ((it + 1) & 1) : ppair;   // this iteration's direction
    const int64_t i0 = (int64_t)B.y + R * threadIdx.x;   // padded rows (an environment's range is a multiple of 4)
    const V alv = pcg_scalar<V>(scal, kAl);
    V rr = V(0), rz = V(0);
    if (i0 < B.z) {
        V pv[4 * R], av[3 * R], rv[3 * R];
        ldv<V, 4 * R>(p + 4 * i0, pv);
        ldv<V, 3 * R>(Ap + 3 * i0, av);
        ldv_rw<V, 3 * R>(r + 3 * i0, rv);
        if constexpr (sizeof(V) == 4) {
            V hv[3 * R], lv[3 * R];
            ldv_rw<V, 3 * R>(xh + 3 * i0, hv);
            ldv_rw<V, 3 * R>(xl + 3 * i0, lv);
#pragma unroll
            for (int a = 0; a < R; ++a)
#pragma unroll
                for (int q = 0; q < 3; ++q) add_pair(hv[3 * a + q], lv[3 * a + q], alv * pv[4 * a + q]);
            stv<V, 3 * R>(xh + 3 * i0, hv);
            stv<V, 3 * R>(xl + 3 * i0, lv);
        } else {
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const int64_t v = prow_v[i0 + a];
                if (v >= 0)
                    for (int q = 0; q < 3; ++q) x[3 * v + q] += (double)alv * (double)pv[4 * a + q];
            }
        }
#pragma unroll
        for (int e = 0; e < 3 * R; ++e) rv[e] -= alv * av[e];
        stv<V, 3 * R>(r + 3 * i0, rv);
        constexpr int ZS = PcgDir<V>::kZs;
        V P[9 * R], zz[ZS * R];
        ldv<V, 9 * R>(Pinv + 9 * i0, P);
#pragma unroll
        for (int a = 0; a < R; ++a) {
            mul33(P + 9 * a, rv[3 * a], rv[3 * a + 1], rv[3 * a + 2], zz + ZS * a);
            if (ZS == 4) zz[ZS * a + ZS - 1] = V(0);
        }
        stv<V, ZS * R>(z + ZS * i0, zz);
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                rr += rv[3 * a + q] * rv[3 * a + q];
                rz += rv[3 * a + q] * zz[ZS * a + q];
            }
    }
    double trr, trz;
    if (last_block_sums<2, V>(rr, rz, part, counters + B.x, B.w, env_nblk[B.x], &trr, &trz) && threadIdx.x == 0) {
        scal[kRr] = trr;
        if (sqrt(trr) <= scal[kThr]) {
            scal[kDone] = 1.0;
            scal[kIters] = (double)(it + 1);
            pcg_ictl(scal)[0] = 1;
        } else {
            scal[kBe] = trz / scal[kRz];
            scal[kRz] = trz;
            pcg_fctl(scal)[1] = (float)scal[kBe];
        }
        // every block read the iteration index and alpha before it arrived
        // at the counter
        scal[kIt] = (double)(it + 1);
        pcg_ictl(scal)[1] = it + 1;
    }
}

// p = z + beta p (FP64 path; z [nvp][3], p [nvp][4]), two rows per thread
template <class V>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_dir(const int4* __restrict__ blk, const V* __restrict__ z, V* __restrict__ p, double* escal) {
    pdl_wait();
    pdl_trigger();
    const int4 B = blk[blockIdx.x];
    double* scal = escal + kEnvScal * B.x;
    if (pcg_ictl(scal)[0] != 0) return;
    const int64_t i0 = (int64_t)B.y + 2 * threadIdx.x;
    if (i0 >= B.z) return;
    const V be = (V)scal[kBe];
    V zv[6], pv[8];
    ldv<V, 6>(z + 3 * i0, zv);
    ldv_rw<V, 8>(p + 4 * i0, pv);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 3; ++q) pv[4 * a + q] = zv[3 * a + q] + be * pv[4 * a + q];
    stv<V, 8>(p + 4 * i0, pv);
}

// ------------------------------------------ PCG of a small environment ---
// One block of kSmallThreads runs the whole solve of one environment of at
// most kSmallRows rows (the multi-block kernels pay two launches and a grid
// of last-block handshakes per iteration, which dominate a system of a few
// hundred rows; with more rows a thread, one SM's latency hiding falls short
// and the multi-block path is faster): the same block-Jacobi PCG with p = 0
// start, stop at
// ||r|| <= rel_tol ||b||, at p^T A p <= 0 (update skipped) or after max_it
// iterations; vectors on the padded rows, the matrix as the multi-block
// SpMV reads it (stored blocks j >= i, transposed blocks j < i), x in FP64.
// Dots per thread and warp in V, across warps in FP64 in a fixed order.
// The environment's scalars are written as the multi-block solve writes
// them, with its stop word set, so the multi-block kernels skip it.
constexpr int kSmallThreads = 512;
constexpr int kSmallRows = kSmallThreads;   // one row a thread: each row's loads are a short chain

template <int NV, class R>
__device__ __forceinline__ void small_sums(R v0, R v1, double* sh, double& t0, double& t1) {
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        if (NV > 1) v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // earlier readers of sh are done
    if (lane == 0) { sh[w] = (double)v0; sh[32 + w] = (double)v1; }
    __syncthreads();
    if (w == 0) {
        double a = lane < kSmallThreads / 32 ? sh[lane] : 0.0;
        double b = lane < kSmallThreads / 32 ? sh[32 + lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            if (NV > 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { sh[64] = a; sh[65] = b; }
    }
    __syncthreads();
    t0 = sh[64];
    t1 = sh[65];
}

// (TA, TP: the matrix and block-inverse storage; V: the vectors; used in
// the FP64 path)
template <class TA, class TP, class V>
__global__ void __launch_bounds__(kSmallThreads)
k_pcg_small(const int4* __restrict__ envs, const int32_t* __restrict__ vprow, const int32_t* __restrict__ rp,
            const int32_t* __restrict__ goff, const int32_t* __restrict__ sci, const int32_t* __restrict__ llen,
            const int32_t* __restrict__ lgoff, const int32_t* __restrict__ lcol, const int32_t* __restrict__ lmir,
            const TA* __restrict__ A, const TP* __restrict__ Pinv, const double* __restrict__ bvec,
            double* __restrict__ xout, V* __restrict__ r, V* __restrict__ z, V* __restrict__ p, V* __restrict__ Ap,
            double* __restrict__ escal, double rel_tol, int max_it) {
    __shared__ double sh[66];
    const int4 E = envs[blockIdx.x];
    double* scal = escal + kEnvScal * E.x;
    // start: x = 0, r = b, z = P^-1 r, p = z
    V lb = V(0), lrz = V(0);
    for (int64_t i = E.y + threadIdx.x; i < E.z; i += kSmallThreads) {
        const int64_t ir = vprow[i];
        const V b0 = (V)bvec[3 * i], b1 = (V)bvec[3 * i + 1], b2 = (V)bvec[3 * i + 2];
        V zz[3];
        const TP* P9 = Pinv + 9 * ir;
        for (int q = 0; q < 3; ++q) zz[q] = (V)P9[3 * q] * b0 + (V)P9[3 * q + 1] * b1 + (V)P9[3 * q + 2] * b2;
        const V bv[3] = {b0, b1, b2};
        for (int q = 0; q < 3; ++q) {
            xout[3 * i + q] = 0.0;
            r[3 * ir + q] = bv[q];
            z[3 * ir + q] = zz[q];
            p[4 * ir + q] = zz[q];
            lb += bv[q] * bv[q];
            lrz += bv[q] * zz[q];
        }
        p[4 * ir + 3] = V(0);
    }
    double bb, rz;
    small_sums<2, V>(lb, lrz, sh, bb, rz);
    const double thr = rel_tol * sqrt(bb);
    int it = 0, done = bb > 0.0 ? 0 : 1, brk = 0;
    while (!done && it < max_it) {
        // Ap and p.Ap (p of the neighbours was written before the last sum's barrier)
        V lpap = V(0);
        for (int64_t i = E.y + threadIdx.x; i < E.z; i += kSmallThreads) {
            const int64_t ir = vprow[i];
            const int64_t g0 = goff[i >> 5];
            const int lane = (int)(i & 31);
            const int ll = llen[i];
            const int len = rp[i + 1] - rp[i] - ll;
            V a0 = V(0), a1 = V(0), a2 = V(0);
            if (ll > 0) {
                const int64_t lg0 = lgoff[i >> 5];
                for (int k = 0; k < ll; ++k) {
                    const int32_t m = lmir[32 * (lg0 + k) + lane];
                    const int64_t j = lcol[32 * (lg0 + k) + lane];
                    TA bt[9];
                    load_blk(A, m >> 5, m & 31, bt);
                    V b[9];
                    for (int q = 0; q < 9; ++q) b[q] = (V)bt[q];
                    const V p0 = p[4 * j], p1 = p[4 * j + 1], p2 = p[4 * j + 2];
                    a0 += b[0] * p0 + b[3] * p1 + b[6] * p2;
                    a1 += b[1] * p0 + b[4] * p1 + b[7] * p2;
                    a2 += b[2] * p0 + b[5] * p1 + b[8] * p2;
                }
            }
            for (int k = 0; k < len; ++k) {
                const int64_t j = sci[32 * (g0 + k) + lane];
                TA bt[9];
                load_blk(A, g0 + k, lane, bt);
                V b[9];
                for (int q = 0; q < 9; ++q) b[q] = (V)bt[q];
                const V p0 = p[4 * j], p1 = p[4 * j + 1], p2 = p[4 * j + 2];
                a0 += b[0] * p0 + b[1] * p1 + b[2] * p2;
                a1 += b[3] * p0 + b[4] * p1 + b[5] * p2;
                a2 += b[6] * p0 + b[7] * p1 + b[8] * p2;
            }
            const V y0 = a0, y1 = a1, y2 = a2;
            Ap[3 * ir] = y0; Ap[3 * ir + 1] = y1; Ap[3 * ir + 2] = y2;
            lpap += p[4 * ir] * y0 + p[4 * ir + 1] * y1 + p[4 * ir + 2] * y2;
        }
        double pap, unused;
        small_sums<1, V>(lpap, V(0), sh, pap, unused);
        if (!(pap > 0.0)) { brk = 1; break; }
        const V alv = (V)(rz / pap);
        const double al = (double)alv;
        V lrr = V(0), lrz2 = V(0);
        for (int64_t i = E.y + threadIdx.x; i < E.z; i += kSmallThreads) {
            const int64_t ir = vprow[i];
            V rv[3], zz[3];
            for (int q = 0; q < 3; ++q) {
                xout[3 * i + q] += al * (double)p[4 * ir + q];
                rv[q] = r[3 * ir + q] - alv * Ap[3 * ir + q];
                r[3 * ir + q] = rv[q];
            }
            const TP* P9 = Pinv + 9 * ir;
            for (int q = 0; q < 3; ++q)
                zz[q] = (V)P9[3 * q] * rv[0] + (V)P9[3 * q + 1] * rv[1] + (V)P9[3 * q + 2] * rv[2];
            for (int q = 0; q < 3; ++q) {
                z[3 * ir + q] = zz[q];
                lrr += rv[q] * rv[q];
                lrz2 += rv[q] * zz[q];
            }
        }
        double rr, rz2;
        small_sums<2, V>(lrr, lrz2, sh, rr, rz2);
        ++it;
        if (sqrt(rr) <= thr) { done = 1; break; }
        const V be = (V)(rz2 / rz);
        rz = rz2;
        for (int64_t i = E.y + threadIdx.x; i < E.z; i += kSmallThreads) {
            const int64_t ir = vprow[i];
            for (int q = 0; q < 3; ++q) p[4 * ir + q] = z[3 * ir + q] + be * p[4 * ir + q];
        }
        __syncthreads();   // p complete before the next product
    }
    if (threadIdx.x == 0) {
        scal[kRz] = rz;
        scal[kBb] = bb;
        scal[kThr] = thr;
        scal[kBreak] = brk ? 1.0 : 0.0;
        scal[kDone] = done ? 1.0 : 0.0;
        scal[kIters] = (double)it;
        scal[kIt] = (double)it;
        pcg_ictl(scal)[0] = 1;   // the multi-block kernels skip this environment
        pcg_ictl(scal)[1] = it;
    }
}

// x = hi + lo in FP64 (mixed path, after the solve), per vertex from its padded row
// (skip: environments solved by k_pcg_small, whose x is already FP64)
__global__ void k_pair_to_f64(int64_t nv, const int32_t* __restrict__ vprow, const float* __restrict__ hi,
                              const float* __restrict__ lo, double* __restrict__ x,
                              const int32_t* __restrict__ vert_env, const int32_t* __restrict__ skip) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    if (skip && skip[vert_env[v]]) return;
    const int64_t r = vprow[v];
    for (int q = 0; q < 3; ++q) x[3 * v + q] = (double)hi[3 * r + q] + (double)lo[3 * r + q];
}

// elementwise products into w (for a fixed-order dot product)
__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = a[i] * b[i];
}

// inertia terms 1/2 m |x + a_j p - xhat|^2 per vertex, layout [na][nv]
__global__ void k_inertia_multi(int64_t nv, const double* __restrict__ x, const double* __restrict__ p,
                                const double* __restrict__ xhat, const double* __restrict__ mass,
                                const double* __restrict__ alphas_env, int astride,
                                const int32_t* __restrict__ vert_env, int na, double* __restrict__ out,
                                const double* __restrict__ fext, double h2, int delta) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double* alphas = alphas_env + (int64_t)astride * vert_env[v];
    const double m = mass[v];
    if (delta) {
        // the change from x: m (a p.(x - xhat) + a^2/2 |p|^2) - h^2 a f.p
        for (int j = 0; j < na; ++j) {
            const double a = alphas[j];
            double e = 0.0, w = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double pc = p[3 * v + c];
                e += m * (a * pc * (x[3 * v + c] - xhat[3 * v + c]) + 0.5 * a * a * pc * pc);
                if (fext) w += a * fext[3 * v + c] * pc;
            }
            out[(int64_t)j * nv + v] = fext ? e - h2 * w : e;
        }
        return;
    }
    for (int j = 0; j < na; ++j) {
        const double a = alphas[j];
        double e = 0.0, w = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double xa = p ? x[3 * v + c] + a * p[3 * v + c] : x[3 * v + c];
            const double d = xa - xhat[3 * v + c];
            e += 0.5 * m * d * d;
            if (fext) w += fext[3 * v + c] * d;
        }
        // external forces (joint step): -h^2 f.(x - xhat) per vertex, the
        // work -h^2 f.x up to a constant of the step (small, so its
        // rounding does not swamp the line search's sufficient-decrease test)
        out[(int64_t)j * nv + v] = fext ? e - h2 * w : e;
    }
}

// E_j = Ein_j + h^2 (Ee_j + Ec_j), per environment (block e, thread j; the
// arrays at stride kES)
__global__ void k_combine(int na, const double* __restrict__ ein, const double* __restrict__ ee,
                          const double* __restrict__ ec, double h2, double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= na) return;
    const int64_t o = (int64_t)kES * blockIdx.x;
    const double c = ec ? ec[o + j] : 0.0;
    out[o + j] = (isfinite(ee[o + j]) && isfinite(c)) ? ein[o + j] + h2 * (ee[o + j] + c) : INFINITY;
}

// segmented sums: block b adds its 2048 elements of segment B.x as
// k_reduce_partial does (8 strided passes of 256 threads, a shuffle tree,
// the eight warp sums); stamp: only entries whose stamp equals *pass.
// blockIdx.y = j sums in[j * in_stride ...] into part[j * gridDim.x ...].
__global__ void k_seg_partial(const double* __restrict__ in, int64_t in_stride, const int4* __restrict__ blk,
                              double* __restrict__ part, const int32_t* __restrict__ stamp,
                              const int32_t* __restrict__ pass) {
    __shared__ double sh[8];
    const int4 B = blk[blockIdx.x];
    in += in_stride * blockIdx.y;
    part += (int64_t)gridDim.x * blockIdx.y;
    const int32_t ps = pass ? *pass : 0;
    double s = 0.0;
    for (int i = 0; i < 8; ++i) {
        const int64_t k = (int64_t)B.y + (int64_t)i * 256 + threadIdx.x;
        if (k < B.z && (!stamp || stamp[k] == ps)) s += in[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}
// one block of 1024 threads per segment (blockIdx.x) and sum j
// (blockIdx.y): the segment's block partials as k_reduce_final sums them,
// into out[out_stride * e + j]
__global__ void k_seg_final(const double* __restrict__ part, int64_t nblk_all,
                            const int32_t* __restrict__ nblk_env, const int32_t* __restrict__ first_blk,
                            double* __restrict__ out, int out_stride) {
    __shared__ double sh[32];
    const int e = blockIdx.x;
    part += nblk_all * blockIdx.y;
    out += blockIdx.y;
    const int nb = nblk_env[e], b0 = first_blk[e];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += 1024) s += part[b0 + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[(int64_t)out_stride * e] = v;
    }
}

// out = x + alpha_env[env] p per vertex of the environments with mask[env]
// != 0 (mask NULL: all); the others get out = x
__global__ void k_axpy_env(int64_t nv, const double* __restrict__ x, const double* __restrict__ p,
                           const double* __restrict__ alpha_env, const int32_t* __restrict__ mask,
                           const int32_t* __restrict__ vert_env, double* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int e = vert_env[v];
    if (mask && !mask[e]) {
        if (out != x)
            for (int c = 0; c < 3; ++c) out[3 * v + c] = x[3 * v + c];
        return;
    }
    const double a = alpha_env[e];
    for (int c = 0; c < 3; ++c) out[3 * v + c] = x[3 * v + c] + a * p[3 * v + c];
}
// v = (x - xt) / h for the vertices of the environments with mask[env] != 0
__global__ void k_velocity_env(int64_t nv, const double* __restrict__ x, const double* __restrict__ xt, double h,
                               const int32_t* __restrict__ mask, const int32_t* __restrict__ vert_env,
                               double* __restrict__ v) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nv || !mask[vert_env[u]]) return;
    for (int c = 0; c < 3; ++c) v[3 * u + c] = (x[3 * u + c] - xt[3 * u + c]) / h;
}
// dst[v] = src[v] for the vertices of the environments with mask[env] != 0
__global__ void k_copy_env(int64_t nv, const double* __restrict__ src, const int32_t* __restrict__ mask,
                           const int32_t* __restrict__ vert_env, double* __restrict__ dst) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !mask[vert_env[v]]) return;
    for (int c = 0; c < 3; ++c) dst[3 * v + c] = src[3 * v + c];
}
// a[v] = 0 for the vertices of the environments with mask[env] == 0
__global__ void k_zero_env(int64_t nv, const int32_t* __restrict__ mask, const int32_t* __restrict__ vert_env,
                           double* __restrict__ a) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || mask[vert_env[v]]) return;
    a[3 * v] = 0.0; a[3 * v + 1] = 0.0; a[3 * v + 2] = 0.0;
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

// segmented fixed-order sums (see SegRed): na sums of R's segments, the
// j-th over in + j in_stride, into out[out_stride e + j]
static cudaError_t seg_sum(Ctx& c, const SegRed& R, const double* in, int64_t in_stride, int na, double* out,
                           int out_stride, const int32_t* stamp = nullptr, const int32_t* pass = nullptr) {
    NewtonState& N = *c.newton;
    if (na < 1) return cudaSuccess;
    if (R.nblk > 0) {
        k_seg_partial<<<dim3((unsigned)R.nblk, (unsigned)na), 256, 0, c.stream>>>(in, in_stride, R.blk.p,
                                                                                 N.seg_part.p, stamp, pass);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    k_seg_final<<<dim3((unsigned)N.n_env, (unsigned)na), 1024, 0, c.stream>>>(N.seg_part.p, R.nblk, R.nblk_env.p,
                                                                             R.first_blk.p, out, out_stride);
    return cudaGetLastError();
}

// the mixed path's view of the elastic tables (pairs) and its input split
static ElasticViewDF df_view(Ctx& c) {
    NewtonState& N = *c.newton;
    auto pair = [](double v) {
        const float h = (float)v;
        return dfl{h, (float)(v - (double)h)};
    };
    return ElasticViewDF{N.ntsys, N.tets.p, reinterpret_cast<const float2*>(N.Dm2.p),
                         reinterpret_cast<const float2*>(N.vol2.p), pair(N.mu), pair(N.lam), pair(1.0 / 3.0),
                         pair(1.0 / 5.0), pair(2.0 / 3.0)};
}
static cudaError_t split_pairs(Ctx& c, const double* v, const double* X, DBuf<float>& hi, DBuf<float>& lo) {
    NewtonState& N = *c.newton;
    k_split_pairs<<<nblk(N.nsys, 256), 256, 0, c.stream>>>(N.nsys, v, X, reinterpret_cast<float4*>(hi.p),
                                                          reinterpret_cast<float4*>(lo.p));
    return cudaGetLastError();
}

cudaError_t nh_eval(Ctx& c, const double* x, bool want_hess) {
    NewtonState& N = *c.newton;
    ElasticView E{N.ntsys, N.tets.p, N.Dminv.p, N.vol.p, N.Xsys.p, N.mu, N.lam};
    if (N.ntsys > 0 && c.P.precision == IPC_PREC_MIXED) {
        GMCP_CUDA_TRY(split_pairs(c, x, N.Xsys.p, N.uh4, N.ul4));
        const unsigned g = nblk(N.ntsys, 128);
        const ElasticViewDF D = df_view(c);
        const float4* uh = reinterpret_cast<const float4*>(N.uh4.p);
        const float4* ul = reinterpret_cast<const float4*>(N.ul4.p);
        float2* tg = reinterpret_cast<float2*>(N.tG.p);
        if (want_hess) k_nh_eval_df<true><<<g, 128, 0, c.stream>>>(D, uh, ul, N.tE.p, tg, N.tH32.p, N.ebad.p, N.tet_env.p);
        else k_nh_eval_df<false><<<g, 128, 0, c.stream>>>(D, uh, ul, N.tE.p, tg, nullptr, N.ebad.p, N.tet_env.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    } else if (N.ntsys > 0) {
        const bool f32 = c.P.precision == IPC_PREC_MIXED;
        const unsigned g = nblk(N.ntsys, 128);
        if (!want_hess)
            k_nh_eval<false, double><<<g, 128, 0, c.stream>>>(E, x, N.tE.p, N.tG.p, nullptr, N.ebad.p, N.tet_env.p);
        else if (f32)
            k_nh_eval<true, float><<<g, 128, 0, c.stream>>>(E, x, N.tE.p, N.tG.p, N.tH32.p, N.ebad.p, N.tet_env.p);
        else
            k_nh_eval<true, double><<<g, 128, 0, c.stream>>>(E, x, N.tE.p, N.tG.p, N.tH64.p, N.ebad.p, N.tet_env.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    return seg_sum(c, N.seg_t, N.tE.p, 0, 1, N.es.p + kEsEe, kES);
}

cudaError_t nh_energy_multi(Ctx& c, const double* x, const double* p, const double* alphas_env, int na, int slot,
                            bool delta) {
    NewtonState& N = *c.newton;
    ElasticView E{N.ntsys, N.tets.p, N.Dminv.p, N.vol.p, N.Xsys.p, N.mu, N.lam};
    if (N.ntsys > 0 && c.P.precision == IPC_PREC_MIXED) {
        GMCP_CUDA_TRY(split_pairs(c, x, N.Xsys.p, N.uh4, N.ul4));
        GMCP_CUDA_TRY(split_pairs(c, p, nullptr, N.ph4, N.pl4));
        k_nh_energy_multi_df<<<nblk(N.ntsys, 128), 128, 0, c.stream>>>(
            df_view(c), reinterpret_cast<const float4*>(N.uh4.p), reinterpret_cast<const float4*>(N.ul4.p),
            reinterpret_cast<const float4*>(N.ph4.p), reinterpret_cast<const float4*>(N.pl4.p), alphas_env, 8,
            N.tet_env.p, na, N.tE8.p, delta ? N.tE.p : nullptr);
        GMCP_CUDA_TRY(cudaGetLastError());
    } else if (N.ntsys > 0) {
        k_nh_energy_multi<<<nblk(N.ntsys, 128), 128, 0, c.stream>>>(E, x, p, alphas_env, 8, N.tet_env.p, na,
                                                                   N.tE8.p, delta ? N.tE.p : nullptr);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    return seg_sum(c, N.seg_t, N.tE8.p, N.ntsys, na, N.es.p + slot, kES);
}

cudaError_t nh_feasible_multi(Ctx& c, const double* x, const double* p, const double* alphas_env, int na,
                              int slot) {
    NewtonState& N = *c.newton;
    ElasticView E{N.ntsys, N.tets.p, N.Dminv.p, N.vol.p, N.Xsys.p, N.mu, N.lam};
    if (N.ntsys > 0 && c.P.precision == IPC_PREC_MIXED) {
        GMCP_CUDA_TRY(split_pairs(c, x, N.Xsys.p, N.uh4, N.ul4));
        GMCP_CUDA_TRY(split_pairs(c, p, nullptr, N.ph4, N.pl4));
        k_nh_feasible_df<<<nblk(N.ntsys, 128), 128, 0, c.stream>>>(
            df_view(c), reinterpret_cast<const float4*>(N.uh4.p), reinterpret_cast<const float4*>(N.ul4.p),
            reinterpret_cast<const float4*>(N.ph4.p), reinterpret_cast<const float4*>(N.pl4.p), alphas_env, 8,
            N.tet_env.p, na, N.tE8.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    } else if (N.ntsys > 0) {
        k_nh_feasible<<<nblk(N.ntsys, 128), 128, 0, c.stream>>>(E, x, p, alphas_env, 8, N.tet_env.p, na, N.tE8.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    return seg_sum(c, N.seg_t, N.tE8.p, N.ntsys, na, N.es.p + slot, kES);
}

cudaError_t assemble_grad(Ctx& c, const double* x, const double* xhat, const void* cgrad, bool cgrad_f32,
                          double* G) {
    NewtonState& N = *c.newton;
    const double h2 = c.prm.h * c.prm.h;
    k_assemble_grad<<<nblk(N.nsys, 256), 256, 0, c.stream>>>(N.nsys, x, xhat, N.mass.p, N.dir.p, N.vte_off.p,
                                                            N.vte.p, N.tG.p, c.P.precision == IPC_PREC_MIXED ? 1 : 0,
                                                            cgrad, cgrad_f32 ? 1 : 0, N.fext, h2,
                                                            G);
    return cudaGetLastError();
}

cudaError_t assemble_bsr(Ctx& c) {
    NewtonState& N = *c.newton;
    const double h2 = c.prm.h * c.prm.h;
    const unsigned g = nblk(32 * N.ngroups, 256);
    if (g == 0) return cudaSuccess;
    if (c.P.precision == IPC_PREC_MIXED)
        k_assemble_sell<float, float, float><<<g, 256, 0, c.stream>>>(
            N.nsys, N.ngroups, N.goff.p, N.gslice.p, N.rp.p, N.llen.p, N.ci.p, N.bt_off.p, N.bt.p, N.tH32.p, N.cmap.p,
            c.cb_val32.p, N.joint ? N.xvals.p : nullptr, N.mass.p, N.dir.p, h2, N.A32.p);
    else
        k_assemble_sell<double, double, double><<<g, 256, 0, c.stream>>>(
            N.nsys, N.ngroups, N.goff.p, N.gslice.p, N.rp.p, N.llen.p, N.ci.p, N.bt_off.p, N.bt.p, N.tH64.p, N.cmap.p,
            c.cb_val64.p, N.joint ? N.xvals.p : nullptr, N.mass.p, N.dir.p, h2, N.A64.p);
    return cudaGetLastError();
}

// dot(a, b) per environment (3 nv entries) into es[slot], fixed order
cudaError_t dot_env(Ctx& c, const double* a, const double* b, int slot) {
    NewtonState& N = *c.newton;
    const int64_t n = 3 * N.nsys;
    k_mul<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, b, N.w.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    return seg_sum(c, N.seg_v3, N.w.p, 0, 1, N.es.p + slot, kES);
}

// Block-Jacobi PCG for A p = b (A on the pattern N.rp / N.ci; FP32 in the
// mixed path, FP64 otherwise), p = 0 start; stops at ||r|| <= rel_tol ||b||,
// at p^T A p <= 0 (that iteration's update is skipped) or after max_it
// iterations.  The host reads the flags once per 16 iterations; kernels
// after the stop return at once.  Returns the iterations taken.
// queue `count` PCG iterations (each kernel returns at once after a stop)
// launch with programmatic stream serialisation (see pdl_wait)
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*k)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPcgThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

template <class TA, class V>
static void pcg_queue(Ctx& c, const TA* A, const V* Pinv, V* r, V* z, V* p, V* Ap, double* xout, V* xh, V* xl,
                      int count) {
    NewtonState& N = *c.newton;
    cudaStream_t s = c.stream;
    const int64_t nvp = N.nvp;
    const unsigned g_row = (unsigned)N.nblk_v, g_multi = (unsigned)N.nblk_p;
    unsigned* cnt_spmv = N.ecount.p + N.n_env;
    unsigned* cnt_upd = N.ecount.p + 2 * N.n_env;
    for (int j = 0; j < count; ++j) {
        launch_pdl(k_pcg_spmv<TA, V>, g_row, s, (const int4*)N.blk_v.p, (const int32_t*)N.env_nblk_v.p,
                   (const int32_t*)N.vprow.p, nvp, (const int32_t*)N.rp.p, (const int32_t*)N.goff.p,
                   (const int32_t*)N.sci.p, (const int32_t*)N.llen.p, (const int32_t*)N.lgoff.p,
                   (const int32_t*)N.lcol.p, (const int32_t*)N.lmir.p, A, p, (const V*)z, Ap, N.part.p, cnt_spmv,
                   N.escal.p);
        launch_pdl(k_pcg_update<V>, g_multi, s, (const int4*)N.blk_p.p, (const int32_t*)N.env_nblk_p.p,
                   (const int32_t*)N.prow_v.p, nvp, Pinv, xout, xh, xl, r, z, (const V*)p, (const V*)Ap, N.part.p,
                   cnt_upd, N.escal.p);
        if (!PcgDir<V>::kFused) launch_pdl(k_pcg_dir<V>, g_multi, s, (const int4*)N.blk_p.p, (const V*)z, p, N.escal.p);
    }
}

static cudaError_t pcg_enqueue_iters(Ctx& c, double* xout, int count) {
    NewtonState& N = *c.newton;
    if (c.P.precision == IPC_PREC_MIXED)
        pcg_queue<float, float>(c, N.A32.p, N.Pinv32.p, N.r32.p, N.z32.p, N.p32.p, N.Ap32.p, xout, N.xh32.p,
                                N.xl32.p, count);
    else
        pcg_queue<double, double>(c, N.A64.p, N.Pinv.p, N.r.p, N.z.p, N.p.p, N.Ap.p, xout, nullptr, nullptr,
                                  count);
    GMCP_CUDA_TRY(cudaGetLastError());
    // every environment's stop flags and iteration count for the host
    return cudaMemcpy2DAsync(N.h_pcg, 4 * sizeof(double), N.escal.p + kBreak, kEnvScal * sizeof(double),
                             3 * sizeof(double), N.n_env, cudaMemcpyDeviceToHost, c.stream);
}

constexpr int kPcgChunk = 16;

// the chunk of kPcgChunk iterations as a CUDA graph (captured on the
// context's private stream); false if capture is not possible
static bool pcg_chunk_graph(Ctx& c, double* xout) {
    NewtonState& N = *c.newton;
    const std::vector<uintptr_t> key = {(uintptr_t)xout, (uintptr_t)N.p.p, (uintptr_t)N.p32.p, (uintptr_t)N.A32.p,
                                        (uintptr_t)N.A64.p, (uintptr_t)N.Ap.p, (uintptr_t)N.Ap32.p,
                                        (uintptr_t)N.r.p, (uintptr_t)N.r32.p, (uintptr_t)N.z.p, (uintptr_t)N.z32.p,
                                        (uintptr_t)N.Pinv.p, (uintptr_t)N.Pinv32.p, (uintptr_t)N.part.p,
                                        (uintptr_t)N.scal.p, (uintptr_t)N.counters.p, (uintptr_t)c.pin,
                                        (uintptr_t)N.xh32.p, (uintptr_t)N.xl32.p, (uintptr_t)N.sci.p,
                                        (uintptr_t)N.goff.p, (uintptr_t)N.llen.p, (uintptr_t)N.lgoff.p,
                                        (uintptr_t)N.lcol.p, (uintptr_t)N.lmir.p, (uintptr_t)N.escal.p,
                                        (uintptr_t)N.ecount.p, (uintptr_t)N.h_pcg, (uintptr_t)N.blk_v.p,
                                        (uintptr_t)N.blk_p.p};
    if (c.pcg_graph.exec && c.pcg_graph.key == key) return true;
    c.pcg_graph.reset();
    if (!c.cap_stream && cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c.cap_stream = nullptr;
        return false;
    }
    cudaStream_t user = c.stream;
    c.stream = c.cap_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = pcg_enqueue_iters(c, xout, kPcgChunk);
        const cudaError_t e2 = cudaStreamEndCapture(c.stream, &g);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    c.stream = user;
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&c.pcg_graph.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c.pcg_graph.reset();
        return false;
    }
    c.pcg_graph.key = key;
    return true;
}

static int64_t nvp_of(const NewtonState& N) { return N.nvp; }

// Block-Jacobi PCG for A p = b (A on the pattern N.rp / N.ci; FP32 matrix
// and vectors in the mixed path, FP64 otherwise; FP64 solution and dots),
// p = 0 start; stops at ||r|| <= rel_tol ||b||, at p^T A p <= 0 (that
// iteration's update is skipped) or after max_it iterations.  The host reads
// the flags once per 16 iterations (a captured graph per chunk when graphs
// are on); kernels after the stop return at once.  Returns the iterations.
cudaError_t pcg_solve(Ctx& c, const double* b, double* xout, double rel_tol, int max_it, int* iters,
                      int* env_iters) {
    NewtonState& N = *c.newton;
    const int64_t nv = N.nsys;
    cudaStream_t s = c.stream;
    const unsigned gr = (unsigned)N.nblk_v;
    if (c.P.precision == IPC_PREC_MIXED) {
        k_diag_inv<float, float><<<nblk(nv, 256), 256, 0, s>>>(nv, N.goff.p, N.A32.p, N.vprow.p, N.Pinv32.p);
        k_pcg_init<float><<<gr, kPcgThreads, 0, s>>>(N.blk_v.p, N.env_nblk_v.p, N.vprow.p, N.Pinv32.p, b, xout,
                                                     N.xh32.p, N.xl32.p, N.r32.p, N.z32.p, N.p32.p, N.part.p,
                                                     N.ecount.p, N.escal.p, rel_tol);
    } else {
        k_diag_inv<double, double><<<nblk(nv, 256), 256, 0, s>>>(nv, N.goff.p, N.A64.p, N.vprow.p, N.Pinv.p);
        k_pcg_init<double><<<gr, kPcgThreads, 0, s>>>(N.blk_v.p, N.env_nblk_v.p, N.vprow.p, N.Pinv.p, b, xout,
                                                      nullptr, nullptr, N.r.p, N.z.p, N.p.p, N.part.p,
                                                      N.ecount.p, N.escal.p, rel_tol);
    }
    GMCP_CUDA_TRY(cudaGetLastError());
    const int ne = N.n_env;
    // small environments: one block each solves the whole system
    if (N.n_small > 0) {
        if (c.P.precision == IPC_PREC_MIXED)
            return cudaErrorInvalidValue;   // not reached: small environments are FP64 only
        else
            k_pcg_small<double, double, double><<<(unsigned)N.n_small, kSmallThreads, 0, s>>>(
                N.small_envs.p, N.vprow.p, N.rp.p, N.goff.p, N.sci.p, N.llen.p, N.lgoff.p, N.lcol.p, N.lmir.p,
                N.A64.p, N.Pinv.p, b, xout, N.sm64.p, N.sm64.p + 3 * nvp_of(N), N.sm64.p + 6 * nvp_of(N),
                N.sm64.p + 10 * nvp_of(N), N.escal.p, rel_tol, max_it);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    const bool large = N.n_small < ne;
    const bool graph = large && c.graphs && !c.prof.on && pcg_chunk_graph(c, xout);
    for (int e = 0; e < ne; ++e) if (env_iters) env_iters[e] = max_it;
    *iters = max_it;
    if (!large) {   // every environment was small: read their scalars once
        GMCP_CUDA_TRY(pcg_enqueue_iters(c, xout, 0));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    for (int it = 0; large && it < max_it;) {
        const int chunk = std::min(kPcgChunk, max_it - it);
        if (graph && chunk == kPcgChunk) GMCP_CUDA_TRY(cudaGraphLaunch(c.pcg_graph.exec, s));
        else GMCP_CUDA_TRY(pcg_enqueue_iters(c, xout, chunk));
        it += chunk;
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
        bool all = true;
        for (int e = 0; e < ne && all; ++e) all = N.h_pcg[4 * e] != 0.0 || N.h_pcg[4 * e + 1] != 0.0;
        if (all) break;
    }
    // iterations: per environment, and the largest (the solve's length)
    int mx = 0;
    for (int e = 0; e < ne; ++e) {
        const bool stopped = N.h_pcg[4 * e] != 0.0 || N.h_pcg[4 * e + 1] != 0.0;
        const int k = stopped ? (int)N.h_pcg[4 * e + 2] : max_it;
        if (env_iters) env_iters[e] = k;
        mx = std::max(mx, k);
    }
    *iters = mx;
    if (c.P.precision == IPC_PREC_MIXED) {
        k_pair_to_f64<<<nblk(nv, 256), 256, 0, s>>>(nv, N.vprow.p, N.xh32.p, N.xl32.p, xout, N.vert_env.p,
                                                    N.n_small > 0 ? N.env_small.p : nullptr);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
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

// blocks of 2048 elements counted from each segment's first element
// (elements scale * off[e] .. scale * off[e + 1])
static cudaError_t build_seg(SegRed& R, const std::vector<int64_t>& off, int64_t scale, cudaStream_t s) {
    const int ne = (int)off.size() - 1;
    std::vector<int4> blk;
    std::vector<int32_t> nb(ne), fb(ne);
    for (int e = 0; e < ne; ++e) {
        const int64_t a = scale * off[e], b = scale * off[e + 1];
        fb[e] = (int32_t)blk.size();
        for (int64_t k = a; k < b; k += 2048)
            blk.push_back(make_int4(e, (int)k, (int)std::min<int64_t>(k + 2048, b), fb[e]));
        nb[e] = (int32_t)blk.size() - fb[e];
    }
    R.nblk = (int64_t)blk.size();
    if (!blk.empty()) GMCP_CUDA_TRY(R.blk.upload(blk.data(), blk.size(), s));
    GMCP_CUDA_TRY(R.nblk_env.upload(nb.data(), nb.size(), s));
    GMCP_CUDA_TRY(R.first_blk.upload(fb.data(), fb.size(), s));
    // host vectors must outlive the copies
    return cudaStreamSynchronize(s);
}

cudaError_t newton_setup(Ctx& c) {
    if (c.newton) return cudaSuccess;
    auto Np = std::make_unique<NewtonState>();
    NewtonState& N = *Np;
    cudaStream_t s = c.stream;
    const ipc_params& q = c.prm;
    // The system: the pad's vertices and tets, followed (joint step with a
    // deformable master) by the master body's.
    const bool joint = c.joint;
    std::vector<double> Xj;
    std::vector<int32_t> Tj;
    std::vector<uint8_t> Dj;
    if (joint) {
        if (c.n_env != 1) return cudaErrorInvalidValue;
        Xj = c.h_X;
        Xj.insert(Xj.end(), c.h_Y0.begin(), c.h_Y0.end());
        Tj = c.h_tets;
        for (int32_t m : c.h_mtets) Tj.push_back(m + (int32_t)c.nv);
        Dj = c.h_dir;
        Dj.insert(Dj.end(), c.h_mdir.begin(), c.h_mdir.end());
    }
    const int64_t nv = joint ? c.nv + c.nmv : c.nv;
    const int64_t nt = joint ? (int64_t)Tj.size() / 4 : c.nt;
    const std::vector<uint8_t>& Dir = joint ? Dj : c.h_dir;
    const std::vector<int64_t> ev = joint ? std::vector<int64_t>{0, nv} : c.env_vert_off;
    const std::vector<int64_t> et = joint ? std::vector<int64_t>{0, nt} : c.env_tet_off;
    N.joint = joint;
    N.nsys = nv;
    N.ntsys = nt;
    N.mu = q.youngs / (2.0 * (1.0 + q.poisson));
    N.lam = q.youngs * q.poisson / ((1.0 + q.poisson) * (1.0 - 2.0 * q.poisson));
    std::vector<double> Dminv(9 * (size_t)nt), vol(nt), mass(nv, 0.0);
    const int32_t* T = joint ? Tj.data() : c.h_tets.data();
    const double* X = joint ? Xj.data() : c.h_X.data();
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* Tt = T + 4 * t;
        double Dm[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) Dm[3 * r + k] = X[3 * Tt[k + 1] + r] - X[3 * Tt[0] + r];
        const double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                           Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
        vol[t] = fabs(det) / 6.0;
        h_inv3(Dm, &Dminv[9 * t]);
        for (int a = 0; a < 4; ++a) mass[Tt[a]] += q.density * vol[t] / 4.0;
    }
    // vertex -> tet corner (t*4+a), increasing tet
    std::vector<int32_t> vte_off(nv + 1, 0), vte(4 * (size_t)nt);
    for (int64_t e = 0; e < 4 * nt; ++e) vte_off[T[e] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vte_off[v + 1] += vte_off[v];
    {
        std::vector<int32_t> cur(vte_off.begin(), vte_off.end() - 1);
        for (int64_t e = 0; e < 4 * nt; ++e) vte[cur[T[e]]++] = (int32_t)e;
    }
    // joint step: every (slave triangle vertex, master triangle vertex) pair
    // whose triangles' rest boxes come within the pattern radius, and the
    // vertex pairs of each master triangle
    std::vector<std::vector<int32_t>> jx(joint ? nv : 0);
    if (joint) {
        const int64_t np = c.nv;
        auto mean_edge = [](const std::vector<int32_t>& F, const double* P) {
            double sum = 0.0;
            int64_t n = 0;
            for (size_t t = 0; t + 2 < F.size(); t += 3)
                for (int a = 0; a < 3; ++a) {
                    const double* u = P + 3 * (int64_t)F[t + a];
                    const double* w = P + 3 * (int64_t)F[t + (a + 1) % 3];
                    sum += sqrt((u[0] - w[0]) * (u[0] - w[0]) + (u[1] - w[1]) * (u[1] - w[1]) + (u[2] - w[2]) * (u[2] - w[2]));
                    ++n;
                }
            return n ? sum / (double)n : 0.0;
        };
        double R = c.joint_radius;
        if (!(R > 0.0))
            R = 2.0 * std::max(mean_edge(c.h_stri, c.h_X.data()), mean_edge(c.h_mtri, c.h_Y0.data())) + 2.0 * c.P.dhat;
        auto box = [](const int32_t* F, const double* P, double* lo, double* hi) {
            for (int q = 0; q < 3; ++q) { lo[q] = INFINITY; hi[q] = -INFINITY; }
            for (int a = 0; a < 3; ++a)
                for (int q = 0; q < 3; ++q) {
                    lo[q] = std::min(lo[q], P[3 * (int64_t)F[a] + q]);
                    hi[q] = std::max(hi[q], P[3 * (int64_t)F[a] + q]);
                }
        };
        std::vector<double> mb(6 * (size_t)c.nmt);
        for (int64_t m = 0; m < c.nmt; ++m) box(&c.h_mtri[3 * m], c.h_Y0.data(), &mb[6 * m], &mb[6 * m + 3]);
        for (int64_t t = 0; t < c.ns; ++t) {
            double lo[3], hi[3];
            box(&c.h_stri[3 * t], c.h_X.data(), lo, hi);
            for (int64_t m = 0; m < c.nmt; ++m) {
                bool near = true;
                for (int q = 0; q < 3; ++q) near = near && lo[q] - R <= mb[6 * m + 3 + q] && mb[6 * m + q] <= hi[q] + R;
                if (!near) continue;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const int32_t u = c.h_stri[3 * t + a], w = (int32_t)np + c.h_mtri[3 * m + b];
                        jx[u].push_back(w);
                        jx[w].push_back(u);
                    }
            }
        }
        for (int64_t m = 0; m < c.nmt; ++m)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) jx[np + c.h_mtri[3 * m + a]].push_back((int32_t)np + c.h_mtri[3 * m + b]);
    }
    // block pattern, row by row: the diagonal, every vertex sharing a tet, and
    // the contact pattern; tb[16 t + 4 a + b] = index of block (T[a], T[b])
    std::vector<int32_t> rp(nv + 1, 0), ci;
    std::vector<int64_t> tb(16 * (size_t)nt);
    ci.reserve(16 * (size_t)nv);
    std::vector<int32_t> row;
    for (int64_t i = 0; i < nv; ++i) {
        row.clear();
        row.push_back((int32_t)i);
        for (int k = vte_off[i]; k < vte_off[i + 1]; ++k) {
            const int64_t t = vte[k] >> 2;
            for (int q = 0; q < 4; ++q) row.push_back(T[4 * t + q]);
        }
        if (i < c.nv)
            for (int k = c.h_cb_row[i]; k < c.h_cb_row[i + 1]; ++k) row.push_back(c.h_cb_col[k]);
        if (joint) row.insert(row.end(), jx[i].begin(), jx[i].end());
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        const int64_t base = (int64_t)ci.size();
        if (base + (int64_t)row.size() >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
        ci.insert(ci.end(), row.begin(), row.end());
        rp[i + 1] = (int32_t)ci.size();
        for (int k = vte_off[i]; k < vte_off[i + 1]; ++k) {
            const int64_t t = vte[k] >> 2;
            const int a = vte[k] & 3;
            for (int q = 0; q < 4; ++q) {
                const int64_t pos = std::lower_bound(row.begin(), row.end(), T[4 * t + q]) - row.begin();
                tb[16 * t + 4 * a + q] = base + pos;
            }
        }
    }
    const int64_t nnzb = (int64_t)ci.size();
    N.nnzb = nnzb;
    // per-block tet contributions in increasing (tet, a, b)
    std::vector<int32_t> bt_off(nnzb + 1, 0), bt(16 * (size_t)nt);
    for (int64_t e = 0; e < 16 * nt; ++e) bt_off[tb[e] + 1]++;
    for (int64_t k = 0; k < nnzb; ++k) bt_off[k + 1] += bt_off[k];
    {
        std::vector<int32_t> cur(bt_off.begin(), bt_off.end() - 1);
        for (int64_t e = 0; e < 16 * nt; ++e) bt[cur[tb[e]]++] = (int32_t)e;
    }
    // global block -> contact block
    std::vector<int32_t> cmap(nnzb, -1);
    for (int64_t i = 0; i < c.nv; ++i)
        for (int k = c.h_cb_row[i]; k < c.h_cb_row[i + 1]; ++k) {
            const int64_t pos = std::lower_bound(ci.begin() + rp[i], ci.begin() + rp[i + 1], c.h_cb_col[k]) - ci.begin();
            cmap[pos] = k;
        }

    // Symmetric sliced-ELL storage.  Row i stores its blocks (i, j), j >= i
    // (the diagonal first), in sliced ELL: slice sl holds rows 32 sl ..
    // 32 sl + 31 and as many groups of 32 blocks as its longest stored row;
    // padding columns are -1.  Its blocks j < i are the transposes of block
    // (j, i), stored in row j: the lower lists give, per row and in column
    // order, j and that block's position (group * 32 + lane).
    const int64_t nslice = (nv + 31) / 32;
    std::vector<int32_t> llen(nv);
    for (int64_t i = 0; i < nv; ++i)
        llen[i] = (int32_t)(std::lower_bound(ci.begin() + rp[i], ci.begin() + rp[i + 1], (int32_t)i) -
                            (ci.begin() + rp[i]));
    std::vector<int32_t> goff(nslice + 1, 0), lgoff(nslice + 1, 0);
    for (int64_t sl = 0; sl < nslice; ++sl) {
        int32_t w = 0, lw = 0;
        for (int64_t i = 32 * sl; i < std::min<int64_t>(nv, 32 * sl + 32); ++i) {
            w = std::max(w, rp[i + 1] - rp[i] - llen[i]);
            lw = std::max(lw, llen[i]);
        }
        if ((int64_t)goff[sl] + w >= ((int64_t)1 << 31) / 288 || (int64_t)lgoff[sl] + lw >= ((int64_t)1 << 26))
            return cudaErrorInvalidValue;
        goff[sl + 1] = goff[sl] + w;
        lgoff[sl + 1] = lgoff[sl] + lw;
    }
    const int64_t ngroups = goff[nslice], nlgroups = lgoff[nslice];
    std::vector<int32_t> gslice(ngroups), sci(32 * (size_t)ngroups, -1);
    std::vector<int32_t> lcol(32 * (size_t)nlgroups + 32, -1), lmir(32 * (size_t)nlgroups + 32, 0);
    for (int64_t sl = 0; sl < nslice; ++sl) {
        for (int32_t g = goff[sl]; g < goff[sl + 1]; ++g) {
            gslice[g] = (int32_t)sl;
            const int k = g - goff[sl];
            for (int lane = 0; lane < 32; ++lane) {
                const int64_t i = 32 * sl + lane;
                if (i < nv && k < rp[i + 1] - rp[i] - llen[i]) sci[32 * (size_t)g + lane] = ci[rp[i] + llen[i] + k];
            }
        }
        for (int32_t g = lgoff[sl]; g < lgoff[sl + 1]; ++g) {
            const int k = g - lgoff[sl];
            for (int lane = 0; lane < 32; ++lane) {
                const int64_t i = 32 * sl + lane;
                if (i >= nv || k >= llen[i]) continue;
                const int32_t j = ci[rp[i] + k];
                const int64_t pos =
                    std::lower_bound(ci.begin() + rp[j], ci.begin() + rp[j + 1], (int32_t)i) - ci.begin();
                if (pos >= rp[j + 1] || ci[pos] != (int32_t)i) return cudaErrorInvalidValue;   // pattern not symmetric
                const int64_t ku = pos - rp[j] - llen[j];
                lcol[32 * (size_t)g + lane] = j;
                lmir[32 * (size_t)g + lane] = (int32_t)((goff[j >> 5] + ku) * 32 + (j & 31));
            }
        }
    }
    N.nslice = nslice;
    N.ngroups = ngroups;
    N.nlgroups = nlgroups;

    // Environments: PCG rows of environment e are padded to a multiple of
    // four and laid out one environment after the other; the PCG kernels'
    // blocks never span two environments (256 vertex rows or 512 padded rows
    // a block, counted from the environment's first row).  With one
    // environment the padded rows are the vertices, padded at the end.
    const int ne = c.n_env;
    N.n_env = ne;
    std::vector<int64_t> poff(ne + 1, 0);
    for (int e = 0; e < ne; ++e) {
        const int64_t n_e = ev[e + 1] - ev[e];
        if (n_e <= 0) return cudaErrorInvalidValue;   // an environment without pad vertices
        poff[e + 1] = poff[e] + (n_e + 3) / 4 * 4;
    }
    const int64_t nvp_env = poff[ne];
    std::vector<int32_t> vprow(nv), prow_v(nvp_env, -1);
    std::vector<int4> blk_v, blk_p;
    N.h_env_nblk_v.assign(ne, 0);
    N.h_env_nblk_p.assign(ne, 0);
    for (int e = 0; e < ne; ++e) {
        const int64_t v0 = ev[e], v1 = ev[e + 1];
        for (int64_t v = v0; v < v1; ++v) {
            vprow[v] = (int32_t)(poff[e] + (v - v0));
            prow_v[poff[e] + (v - v0)] = (int32_t)v;
        }
        const int first_v = (int)blk_v.size(), first_p = (int)blk_p.size();
        for (int64_t r = v0; r < v1; r += kPcgThreads)
            blk_v.push_back(make_int4(e, (int)r, (int)std::min<int64_t>(r + kPcgThreads, v1), first_v));
        for (int64_t r = poff[e]; r < poff[e + 1]; r += 2 * kPcgThreads)
            blk_p.push_back(make_int4(e, (int)r, (int)std::min<int64_t>(r + 2 * kPcgThreads, poff[e + 1]), first_p));
        N.h_env_nblk_v[e] = (int32_t)blk_v.size() - first_v;
        N.h_env_nblk_p[e] = (int32_t)blk_p.size() - first_p;
    }
    N.nblk_v = (int64_t)blk_v.size();
    N.nblk_p = (int64_t)blk_p.size();
    {
        // small environments (by their own size only, so a batch solves each
        // environment as a context holding it alone would); FP64 path only:
        // with the FP32 matrix the one-block solve stalled on the joint patch
        // test where the multi-block FP32 solve converges, so the mixed path
        // keeps the multi-block kernels
        std::vector<int4> small;
        std::vector<int32_t> flag(ne, 0);
        const bool f64 = c.P.precision != IPC_PREC_MIXED;
        for (int e = 0; e < ne; ++e)
            if (f64 && ev[e + 1] - ev[e] <= kSmallRows) {
                small.push_back(make_int4(e, (int)ev[e], (int)ev[e + 1], 0));
                flag[e] = 1;
            }
        N.n_small = (int64_t)small.size();
        GMCP_CUDA_TRY(N.env_small.upload(flag.data(), flag.size(), s));
        if (!small.empty()) GMCP_CUDA_TRY(N.small_envs.upload(small.data(), small.size(), s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // the SpMV reads the direction at the padded rows of its columns
    for (auto& col : sci) if (col >= 0) col = vprow[col];
    for (auto& col : lcol) if (col >= 0) col = vprow[col];
    GMCP_CUDA_TRY(N.vprow.upload(vprow.data(), vprow.size(), s));
    GMCP_CUDA_TRY(N.prow_v.upload(prow_v.data(), prow_v.size(), s));
    GMCP_CUDA_TRY(N.blk_v.upload(blk_v.data(), blk_v.size(), s));
    GMCP_CUDA_TRY(N.blk_p.upload(blk_p.data(), blk_p.size(), s));
    GMCP_CUDA_TRY(N.env_nblk_v.upload(N.h_env_nblk_v.data(), ne, s));
    GMCP_CUDA_TRY(N.env_nblk_p.upload(N.h_env_nblk_p.data(), ne, s));
    GMCP_CUDA_TRY(N.escal.ensure((size_t)kEnvScal * ne));
    GMCP_CUDA_TRY(cudaMemsetAsync(N.escal.p, 0, sizeof(double) * kEnvScal * ne, s));
    GMCP_CUDA_TRY(N.ecount.ensure(3 * (size_t)ne));
    GMCP_CUDA_TRY(cudaMemsetAsync(N.ecount.p, 0, sizeof(unsigned) * 3 * ne, s));
    if (cudaMallocHost(reinterpret_cast<void**>(&N.h_pcg), sizeof(double) * 4 * ne) != cudaSuccess)
        return cudaErrorMemoryAllocation;

    // The Newton iteration per environment: the environment of each vertex
    // and tet, segmented sums over vertices (1 and 3 entries each), tets and
    // slave triangles, the per-environment scalars, flags and step sizes, and
    // pinned host copies of them.
    if (et[ne] != nt || c.env_stri_off[ne] != c.ns || 3 * nv > INT32_MAX) return cudaErrorInvalidValue;
    {
        std::vector<int32_t> venv(nv), tenv(nt);
        N.h_lbar.assign(ne, 0.0);
        N.h_has_dir.assign(ne, 0);
        N.h_dir_surf.assign(ne, 0);
        for (int e = 0; e < ne; ++e) {
            for (int64_t v = ev[e]; v < ev[e + 1]; ++v) {
                venv[v] = e;
                if (Dir[v]) N.h_has_dir[e] = 1;
            }
            double ve = 0.0;   // the order of the whole-scene sum, over this environment's tets
            for (int64_t t = et[e]; t < et[e + 1]; ++t) {
                tenv[t] = e;
                ve += vol[t];
            }
            const int64_t nte = et[e + 1] - et[e];
            N.h_lbar[e] = nte > 0 ? cbrt(ve / (double)nte) : 0.0;
        }
        // Dirichlet vertices on a contact surface (else their motion alone
        // moves no contact primitive, and its step bound is 1)
        for (int64_t t = 0; t < c.ns; ++t)
            for (int a = 0; a < 3; ++a) {
                const int32_t v = c.h_stri[3 * t + a];
                if (Dir[v]) N.h_dir_surf[venv[v]] = 1;
            }
        if (joint)
            for (int64_t m = 0; m < c.nmt; ++m)
                for (int a = 0; a < 3; ++a) {
                    const int64_t v = c.nv + c.h_mtri[3 * m + a];
                    if (Dir[v]) N.h_dir_surf[venv[v]] = 1;
                }
        GMCP_CUDA_TRY(N.vert_env.upload(venv.data(), venv.size(), s));
        GMCP_CUDA_TRY(N.tet_env.upload(tenv.data(), tenv.size(), s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    GMCP_CUDA_TRY(build_seg(N.seg_v, ev, 1, s));
    GMCP_CUDA_TRY(build_seg(N.seg_v3, ev, 3, s));
    GMCP_CUDA_TRY(build_seg(N.seg_t, et, 1, s));
    GMCP_CUDA_TRY(build_seg(N.seg_s, c.env_stri_off, 1, s));
    const int64_t seg_max = std::max(std::max(N.seg_v.nblk, N.seg_v3.nblk), std::max(N.seg_t.nblk, N.seg_s.nblk));
    GMCP_CUDA_TRY(N.seg_part.ensure(8 * (size_t)seg_max + 8));
    GMCP_CUDA_TRY(N.es.ensure((size_t)kES * ne));
    GMCP_CUDA_TRY(cudaMemsetAsync(N.es.p, 0, sizeof(double) * kES * ne, s));
    GMCP_CUDA_TRY(N.ebad.ensure((size_t)ne));
    GMCP_CUDA_TRY(N.ealpha.ensure((size_t)ne));
    GMCP_CUDA_TRY(N.eal.ensure(8 * (size_t)ne));
    GMCP_CUDA_TRY(N.emask.ensure(4 * (size_t)ne));
    GMCP_CUDA_TRY(N.ebits.ensure(2 * (size_t)ne));
    GMCP_CUDA_TRY(N.ezero.ensure(1));
    GMCP_CUDA_TRY(cudaMemsetAsync(N.ezero.p, 0, sizeof(double), s));
    {
        const size_t bytes = sizeof(double) * ((size_t)kES + 8 + 1) * ne + sizeof(unsigned long long) * 2 * ne +
                             sizeof(int32_t) * 5 * ne;
        if (cudaMallocHost(&N.h_pin, bytes) != cudaSuccess) return cudaErrorMemoryAllocation;
        char* q = (char*)N.h_pin;
        N.h_es = (double*)q;                 q += sizeof(double) * kES * ne;
        N.h_eal = (double*)q;                q += sizeof(double) * 8 * ne;
        N.h_ealpha = (double*)q;             q += sizeof(double) * ne;
        N.h_ebits = (unsigned long long*)q;  q += sizeof(unsigned long long) * 2 * ne;
        N.h_emask = (int32_t*)q;             q += sizeof(int32_t) * 4 * ne;
        N.h_ebad = (int32_t*)q;
    }

    const size_t n3 = 3 * (size_t)nv;
    GMCP_CUDA_TRY(N.goff.upload(goff.data(), goff.size(), s));
    GMCP_CUDA_TRY(N.gslice.upload(gslice.data(), gslice.size(), s));
    GMCP_CUDA_TRY(N.sci.upload(sci.data(), sci.size(), s));
    GMCP_CUDA_TRY(N.llen.upload(llen.data(), llen.size(), s));
    GMCP_CUDA_TRY(N.lgoff.upload(lgoff.data(), lgoff.size(), s));
    GMCP_CUDA_TRY(N.lcol.upload(lcol.data(), lcol.size(), s));
    GMCP_CUDA_TRY(N.lmir.upload(lmir.data(), lmir.size(), s));
    GMCP_CUDA_TRY(N.tets.upload(T, 4 * (size_t)nt, s));
    GMCP_CUDA_TRY(N.Dminv.upload(Dminv.data(), Dminv.size(), s));
    GMCP_CUDA_TRY(N.vol.upload(vol.data(), vol.size(), s));
    GMCP_CUDA_TRY(N.mass.upload(mass.data(), mass.size(), s));
    GMCP_CUDA_TRY(N.dir.upload(Dir.data(), Dir.size(), s));
    GMCP_CUDA_TRY(N.Xsys.upload(X, 3 * (size_t)nv, s));
    if (joint) {
        GMCP_CUDA_TRY(N.xvals.ensure(9 * (size_t)nnzb + 9));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.xvals.p, 0, sizeof(double) * (9 * (size_t)nnzb + 9), s));
    }
    GMCP_CUDA_TRY(N.vte_off.upload(vte_off.data(), vte_off.size(), s));
    GMCP_CUDA_TRY(N.vte.upload(vte.data(), vte.size(), s));
    GMCP_CUDA_TRY(N.rp.upload(rp.data(), rp.size(), s));
    GMCP_CUDA_TRY(N.ci.upload(ci.data(), ci.size(), s));
    GMCP_CUDA_TRY(N.bt_off.upload(bt_off.data(), bt_off.size(), s));
    GMCP_CUDA_TRY(N.bt.upload(bt.data(), bt.size(), s));
    GMCP_CUDA_TRY(N.cmap.upload(cmap.data(), cmap.size(), s));
    GMCP_CUDA_TRY(N.tE.ensure((size_t)nt + 1));
    GMCP_CUDA_TRY(N.tG.ensure(12 * (size_t)nt + 12));
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    if (f32) {
        // Dm^-1 and the volumes as pairs, the input splits' buffers
        std::vector<float> dm2(18 * (size_t)nt + 18), vol2(2 * (size_t)nt + 2);
        auto put = [](float* d, double v) {
            const float h = (float)v;
            d[0] = h;
            d[1] = (float)(v - (double)h);
        };
        for (size_t k = 0; k < 9 * (size_t)nt; ++k) put(&dm2[2 * k], Dminv[k]);
        for (size_t k = 0; k < (size_t)nt; ++k) put(&vol2[2 * k], vol[k]);
        GMCP_CUDA_TRY(N.Dm2.upload(dm2.data(), dm2.size(), s));
        GMCP_CUDA_TRY(N.vol2.upload(vol2.data(), vol2.size(), s));
        for (DBuf<float>* b : {&N.uh4, &N.ul4, &N.ph4, &N.pl4}) GMCP_CUDA_TRY(b->ensure(4 * (size_t)nv + 4));
    }
    if (f32) GMCP_CUDA_TRY(N.tH32.ensure(HBlk<float>::kPerTet * ((size_t)nt + 1)));
    else GMCP_CUDA_TRY(N.tH64.ensure(HBlk<double>::kPerTet * ((size_t)nt + 1)));
    GMCP_CUDA_TRY(N.tE8.ensure(8 * (size_t)nt + 8));
    // PCG vectors: rows padded per environment (above), the padding zero
    const int64_t nvp = nvp_env;
    if (N.n_small > 0) GMCP_CUDA_TRY(N.sm64.ensure(13 * (size_t)nvp + 16));
    N.nvp = nvp;
    if (f32) {
        GMCP_CUDA_TRY(N.A32.ensure(288 * (size_t)ngroups + 288));
        for (DBuf<float>* b : {&N.r32, &N.Ap32, &N.xh32, &N.xl32}) {
            GMCP_CUDA_TRY(b->ensure(3 * (size_t)nvp));
            GMCP_CUDA_TRY(cudaMemsetAsync(b->p, 0, sizeof(float) * 3 * nvp, s));
        }
        GMCP_CUDA_TRY(N.z32.ensure(4 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.z32.p, 0, sizeof(float) * 4 * nvp, s));
        GMCP_CUDA_TRY(N.p32.ensure(8 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.p32.p, 0, sizeof(float) * 8 * nvp, s));
        GMCP_CUDA_TRY(N.Pinv32.ensure(9 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.Pinv32.p, 0, sizeof(float) * 9 * nvp, s));
    } else {
        GMCP_CUDA_TRY(N.A64.ensure(288 * (size_t)ngroups + 288));
        for (DBuf<double>* b : {&N.r, &N.Ap}) {
            GMCP_CUDA_TRY(b->ensure(3 * (size_t)nvp));
            GMCP_CUDA_TRY(cudaMemsetAsync(b->p, 0, sizeof(double) * 3 * nvp, s));
        }
        GMCP_CUDA_TRY(N.z.ensure(3 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.z.p, 0, sizeof(double) * 3 * nvp, s));
        GMCP_CUDA_TRY(N.p.ensure(4 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.p.p, 0, sizeof(double) * 4 * nvp, s));
        GMCP_CUDA_TRY(N.Pinv.ensure(9 * (size_t)nvp));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.Pinv.p, 0, sizeof(double) * 9 * nvp, s));
    }
    GMCP_CUDA_TRY(N.part.ensure(2 * (size_t)std::max(N.nblk_v, N.nblk_p) + 2));
    GMCP_CUDA_TRY(N.counters.ensure(4));
    GMCP_CUDA_TRY(cudaMemsetAsync(N.counters.p, 0, 4 * sizeof(unsigned), s));
    for (DBuf<double>* b : {&N.w, &N.xhat, &N.xt, &N.G, &N.dirn, &N.tmp, &N.P, &N.dP, &N.xi, &N.xl})
        GMCP_CUDA_TRY(b->ensure(n3));
    if (f32) GMCP_CUDA_TRY(N.cgrad32.ensure(n3));
    else GMCP_CUDA_TRY(N.cgrad64.ensure(n3));
    GMCP_CUDA_TRY(N.xm.ensure(3 * (size_t)c.nmv + 3));
    GMCP_CUDA_TRY(N.dxm.ensure(3 * (size_t)c.nmv + 3));
    if (c.nmv > 0)
        GMCP_CUDA_TRY(cudaMemcpyAsync(N.xm.p, c.Y0.p, sizeof(double) * 3 * c.nmv, cudaMemcpyDeviceToDevice, s));
    GMCP_CUDA_TRY(N.ein8.ensure(8 * (size_t)nv));
    GMCP_CUDA_TRY(N.triE8.ensure(8 * (size_t)c.ns + 8));
    GMCP_CUDA_TRY(N.scal.ensure(64));
    // host vectors must outlive the asynchronous copies
    GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    c.newton = std::move(Np);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// energies and the assembled system
// ---------------------------------------------------------------------------
// the master positions that belong to system positions x: the master rows
// of x in the joint step, else the context's kinematic master
const double* master_of(Ctx& c, const double* x) {
    return c.newton->joint ? x + 3 * c.nv : c.newton->xm.p;
}
const double* master_dir_of(Ctx& c, const double* p) {
    return c.newton->joint ? p + 3 * c.nv : nullptr;
}

// The master entries of the samples at (x, xm), sorted by destination and
// summed in a fixed order (see k_ml_reduce): the rows, and with xvals the
// blocks.  Uses the context's entry buffers (grown and retried when the
// entries outnumber them).
cudaError_t sorted_master_terms(Ctx& c, const double* x, const double* xm, int64_t nrows, int64_t row_base,
                                void* rows_out, bool rows_f32, const int32_t* rp, const int32_t* llen,
                                const int32_t* ci, double* xvals, bool* miss) {
    cudaStream_t s = c.stream;
    if (c.ml_cap == 0) c.ml_cap = std::max<int64_t>((int64_t)1 << 16, 64 * c.ns);
    for (int attempt = 0;; ++attempt) {
        GMCP_CUDA_TRY(c.ml_ij.ensure(2 * (size_t)c.ml_cap));
        GMCP_CUDA_TRY(c.ml_blk.ensure(9 * (size_t)c.ml_cap));
        GMCP_CUDA_TRY(c.ml_perm.ensure((size_t)c.ml_cap));
        GMCP_CUDA_TRY(c.ml_count.ensure(1));
        GMCP_CUDA_TRY(contact_master_hess(c, x, xm, c.ml_ij.p, c.ml_blk.p, c.ml_cap, c.ml_count.p, true,
                                          xvals != nullptr));
        unsigned long long need = 0;
        GMCP_CUDA_TRY(cudaMemcpyAsync(&need, c.ml_count.p, sizeof(need), cudaMemcpyDeviceToHost, s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
        if ((int64_t)need <= c.ml_cap) break;
        if (attempt >= 2) return cudaErrorInvalidValue;
        c.ml_cap = (int64_t)need + (int64_t)need / 2 + 1024;
    }
    GMCP_CUDA_TRY(c.ml_cnt.ensure((size_t)nrows + 1));
    GMCP_CUDA_TRY(c.ml_off.ensure((size_t)nrows + 2));
    GMCP_CUDA_TRY(c.ml_cur.ensure((size_t)nrows + 1));
    GMCP_CUDA_TRY(c.ml_tmp.ensure(2 * scan_tmp_size(nrows + 1)));
    GMCP_CUDA_TRY(c.ml_err.ensure(1));
    GMCP_CUDA_TRY(cudaMemsetAsync(c.ml_cnt.p, 0, sizeof(int32_t) * (nrows + 1), s));
    GMCP_CUDA_TRY(cudaMemsetAsync(c.ml_cur.p, 0, sizeof(int32_t) * (nrows + 1), s));
    GMCP_CUDA_TRY(cudaMemsetAsync(c.ml_err.p, 0, sizeof(int32_t), s));
    const unsigned g = (unsigned)std::min<int64_t>(4096, (c.ml_cap + 255) / 256);
    k_ml_count<<<g, 256, 0, s>>>(c.ml_ij.p, c.ml_count.p, c.ml_cap, nrows, c.ml_cnt.p, c.ml_err.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(exclusive_scan_i32(c.ml_cnt.p, c.ml_off.p, nrows + 1, c.ml_tmp.p, c.ml_tmp.n, s));
    k_ml_fill<<<g, 256, 0, s>>>(c.ml_ij.p, c.ml_count.p, c.ml_cap, nrows, c.ml_off.p, c.ml_cur.p, c.ml_perm.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (rows_f32)
        k_ml_reduce<float><<<nblk(nrows, 128), 128, 0, s>>>(nrows, c.ml_off.p, c.ml_perm.p, c.ml_ij.p, c.ml_blk.p, rp,
                                                           llen, ci, xvals, (float*)rows_out, row_base, c.ml_err.p);
    else
        k_ml_reduce<double><<<nblk(nrows, 128), 128, 0, s>>>(nrows, c.ml_off.p, c.ml_perm.p, c.ml_ij.p, c.ml_blk.p,
                                                            rp, llen, ci, xvals, (double*)rows_out, row_base,
                                                            c.ml_err.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    int32_t err = 0;
    GMCP_CUDA_TRY(cudaMemcpyAsync(&err, c.ml_err.p, sizeof(err), cudaMemcpyDeviceToHost, s));
    GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    if (miss) *miss = err != 0;
    return err ? cudaErrorInvalidValue : cudaSuccess;
}

// Joint step: the gradient rows of the master vertices (into the contact
// gradient's rows nv .. nsys) and, with want_hess, the blocks with master
// vertices (into xvals), from the samples of the last pass at x.  A block
// outside the pattern sets N.joint_miss and fails the call.
cudaError_t joint_master_terms(Ctx& c, const double* x, bool want_hess) {
    NewtonState& N = *c.newton;
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    const size_t gb = f32 ? sizeof(float) : sizeof(double);
    char* cg = f32 ? (char*)N.cgrad32.p : (char*)N.cgrad64.p;
    GMCP_CUDA_TRY(cudaMemsetAsync(cg + gb * 3 * c.nv, 0, gb * 3 * (N.nsys - c.nv), c.stream));
    if (want_hess) GMCP_CUDA_TRY(cudaMemsetAsync(N.xvals.p, 0, sizeof(double) * 9 * N.nnzb, c.stream));
    bool miss = false;
    const cudaError_t e = sorted_master_terms(c, x, x + 3 * c.nv, N.nsys, 0, cg, f32, N.rp.p, N.llen.p, N.ci.p,
                                              want_hess ? N.xvals.p : nullptr, &miss);
    if (miss) N.joint_miss = true;
    return e;
}

// change of each environment's incremental potential from x to x +
// alphas_env[8 e + j] p, j < na (<= 8), into es[kEsE8 + j] (reading R22:
// every term's change is formed before the sums -- per tet, per vertex, per
// sample -- so the sufficient-decrease test is not lost in the rounding of
// the total); the contact term is the frozen-linear potential of the samples
// active at x (requires the candidate lists and per-tet energies of x, i.e.
// the system assembled at x).  ee0: alphas_env[8 e] = 0, whose change is 0.
cudaError_t energy_batch(Ctx& c, const double* x, const double* p, const double* alphas_env, int na,
                         bool with_contact, bool ee0) {
    NewtonState& N = *c.newton;
    double* es = N.es.p;
    const int ne = N.n_env;
    if (ee0 && na > 1) {
        // slot 0 is alpha = 0: no change
        GMCP_CUDA_TRY(nh_energy_multi(c, x, p, alphas_env + 1, na - 1, kEsEe8 + 1, true));
        GMCP_CUDA_TRY(cudaMemset2DAsync(es + kEsEe8, kES * sizeof(double), 0, sizeof(double), ne, c.stream));
    } else {
        GMCP_CUDA_TRY(nh_energy_multi(c, x, p, alphas_env, na, kEsEe8, true));
    }
    const double h2 = c.prm.h * c.prm.h;
    k_inertia_multi<<<nblk(N.nsys, 256), 256, 0, c.stream>>>(N.nsys, x, p, N.xhat.p, N.mass.p, alphas_env, 8,
                                                             N.vert_env.p, na, N.ein8.p, N.fext, h2, 1);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(seg_sum(c, N.seg_v, N.ein8.p, N.nsys, na, es + kEsEin8, kES));
    if (with_contact) {
        GMCP_CUDA_TRY(contact_lagged(c, x, master_of(c, x), p, alphas_env, na, N.triE8.p, nullptr, 8,
                                     N.joint ? p + 3 * c.nv : nullptr));
        GMCP_CUDA_TRY(seg_sum(c, N.seg_s, N.triE8.p, c.ns, na, es + kEsEc8, kES));
    }
    k_combine<<<ne, 32, 0, c.stream>>>(na, es + kEsEin8, es + kEsEe8, with_contact ? es + kEsEc8 : nullptr, h2,
                                       es + kEsE8);
    return cudaGetLastError();
}

// per environment: contact and elastic potentials es[kEsEc], es[kEsEe], the
// total es[kEsE] and |G|^2 es[kEsG2] at x, the gradient G (Dirichlet rows
// zero), optionally the matrix A; inverted-tet flags in N.ebad.  The broad
// phase runs at (x, current master).
cudaError_t assemble_system(Ctx& c, const double* x, int hess) {
    NewtonState& N = *c.newton;
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    double* es = N.es.p;
    const int ne = N.n_env;
    GMCP_CUDA_TRY(cudaMemsetAsync(N.ebad.p, 0, sizeof(int32_t) * ne, c.stream));
    {
        ProfScope ps(c.prof, c.stream, "elastic");
        GMCP_CUDA_TRY(nh_eval(c, x, hess == kHessAll));
    }
    const double* xm = master_of(c, x);
    GMCP_CUDA_TRY(run_candidates(c, x, xm));
    void* cg = f32 ? (void*)N.cgrad32.p : (void*)N.cgrad64.p;
    GMCP_CUDA_TRY(contact_eval(c, x, xm, nullptr, cg, hess != kHessNone, nullptr));
    // the contact energy of the samples of this pass (stamped triangles)
    GMCP_CUDA_TRY(seg_sum(c, N.seg_s, c.tri_E.p, 0, 1, es + kEsEc, kES, c.tri_stamp.p, c.misc_i32.p + kSlotPass));
    if (N.joint) GMCP_CUDA_TRY(joint_master_terms(c, x, hess != kHessNone));
    {
        ProfScope ps(c.prof, c.stream, "assemble");
        GMCP_CUDA_TRY(assemble_grad(c, x, N.xhat.p, cg, f32, N.G.p));
        if (hess == kHessAll) GMCP_CUDA_TRY(assemble_bsr(c));
    }
    // total energy: inertia at x (one term, alpha 0, p unused)
    const double h2 = c.prm.h * c.prm.h;
    k_inertia_multi<<<nblk(N.nsys, 256), 256, 0, c.stream>>>(N.nsys, x, nullptr, N.xhat.p, N.mass.p, N.ezero.p, 0,
                                                             N.vert_env.p, 1, N.ein8.p, N.fext, h2, 0);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(seg_sum(c, N.seg_v, N.ein8.p, 0, 1, es + kEsEin, kES));
    k_combine<<<ne, 32, 0, c.stream>>>(1, es + kEsEin, es + kEsEe, es + kEsEc, h2, es + kEsE);
    GMCP_CUDA_TRY(cudaGetLastError());
    return dot_env(c, N.G.p, N.G.p, kEsG2);
}

// the elastic Hessian blocks at x and the global matrix, after an
// assemble_system(c, x, kHessContact) (the contact and master blocks are
// already in place)
cudaError_t finish_hessian(Ctx& c, const double* x) {
    NewtonState& N = *c.newton;
    if (N.ntsys > 0) {
        ProfScope ps(c.prof, c.stream, "elastic");
        const unsigned g = nblk(N.ntsys, 128);
        if (c.P.precision == IPC_PREC_MIXED) {
            GMCP_CUDA_TRY(split_pairs(c, x, N.Xsys.p, N.uh4, N.ul4));
            k_nh_hess_df<<<g, 128, 0, c.stream>>>(df_view(c), reinterpret_cast<const float4*>(N.uh4.p),
                                                  reinterpret_cast<const float4*>(N.ul4.p), N.tH32.p);
        } else {
            ElasticView E{N.ntsys, N.tets.p, N.Dminv.p, N.vol.p, N.Xsys.p, N.mu, N.lam};
            k_nh_hess64<<<g, 128, 0, c.stream>>>(E, x, N.tH64.p);
        }
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    ProfScope ps(c.prof, c.stream, "assemble");
    return assemble_bsr(c);
}

// ------------------------------------------------- per-environment vectors ---
cudaError_t vec_axpy_env(Ctx& c, const double* x, const double* p, const double* alpha_env, const int32_t* mask,
                         double* out) {
    NewtonState& N = *c.newton;
    k_axpy_env<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, x, p, alpha_env, mask, N.vert_env.p, out);
    return cudaGetLastError();
}
cudaError_t vec_copy_env(Ctx& c, const double* src, const int32_t* mask, double* dst) {
    NewtonState& N = *c.newton;
    k_copy_env<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, src, mask, N.vert_env.p, dst);
    return cudaGetLastError();
}
cudaError_t vec_zero_env(Ctx& c, const int32_t* mask, double* a) {
    NewtonState& N = *c.newton;
    k_zero_env<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, mask, N.vert_env.p, a);
    return cudaGetLastError();
}
cudaError_t vec_copy_master_env(Ctx& c, const double* src, const int32_t* mask, double* dst) {
    if (c.nmv == 0) return cudaSuccess;
    k_copy_env<<<nblk(c.nmv, 256), 256, 0, c.stream>>>(c.nmv, src, mask, c.mvert_env.p, dst);
    return cudaGetLastError();
}
cudaError_t vec_velocity_env(Ctx& c, const double* x, const double* xt, const int32_t* mask, double* v) {
    NewtonState& N = *c.newton;
    k_velocity_env<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, x, xt, c.prm.h, mask, N.vert_env.p, v);
    return cudaGetLastError();
}

// --------------------------------------------------------------- vectors ---
cudaError_t vec_axpy(Ctx& c, int64_t n, double a, const double* x, const double* p, double* out) {
    k_axpy<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, x, p, out);
    return cudaGetLastError();
}
cudaError_t vec_xhat(Ctx& c, const double* x, const double* v, double* xhat) {
    const double* g = c.prm.gravity;
    k_xhat<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, x, v, c.prm.h, g[0], g[1], g[2], xhat);
    return cudaGetLastError();
}
cudaError_t vec_dir_delta(Ctx& c, const double* x, const double* xhat, double* dP) {
    k_dir_delta<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, c.newton->dir.p, x, xhat, dP);
    return cudaGetLastError();
}
cudaError_t vec_set_dir(Ctx& c, const double* src, double* dst) {
    k_set_dir<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, c.newton->dir.p, src, dst);
    return cudaGetLastError();
}
cudaError_t vec_free_delta(Ctx& c, const double* P, const double* xi, double* dP) {
    k_free_delta<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, c.newton->dir.p, P, xi, dP);
    return cudaGetLastError();
}
cudaError_t vec_zero_dir(Ctx& c, double* p) {
    k_zero_dir<<<nblk(c.newton->nsys, 256), 256, 0, c.stream>>>(c.newton->nsys, c.newton->dir.p, p);
    return cudaGetLastError();
}
cudaError_t vec_velocity(Ctx& c, const double* x, const double* xt, double* v) {
    const int64_t n = 3 * c.newton->nsys;
    k_velocity<<<nblk(n, 256), 256, 0, c.stream>>>(n, x, xt, c.prm.h, v);
    return cudaGetLastError();
}
cudaError_t vec_neg(Ctx& c, int64_t n, const double* a, double* out) {
    k_neg<<<nblk(n, 256), 256, 0, c.stream>>>(n, a, out);
    return cudaGetLastError();
}

}  // namespace gmcp
