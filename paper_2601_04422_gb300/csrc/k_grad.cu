// Reverse-mode gradient of an energy through the layered MPS simulation (tnsim_grad).
//
// Conventions: for a complex intermediate X the kernels carry Xb = dE/d(conj X), so
// that dE = 2 Re <Xb, dX>.  The forward is the library's own layer path; the
// backward of one two-qubit update (k_gate_bwd, one CTA per gate) follows the
// chain rule of its steps:
//   right site c Y (Y = U^H T, c = |T|_F / |Y|_F):  Yb = c Bb - (dc c / 2K2) Y,
//     dc = 2 Re <Bb, Y>, plus (dc c / 2F2) T into Tb;
//   kept subspace of T (the left site U; the loss depends on U only through
//   span(U) because a gauge change U R, R^H Y leaves the state unchanged):
//     Tb += U Yb + (I - P) Ut S_k^-2 Y + (Z + Z^H) T,   Ut = Ub + T Yb^H,
//     Z = U_D (G o (U_D^H Ut)) U^H,  G_lj = 1 / (s_j^2 - s_l^2) across the cut,
//     P the projector on the nonzero singular directions (columns of the Jacobi
//     matrix W divided by their norms), U_D the discarded nonzero ones; (I - P) Ut is
//     formed as (I - P) Ub (equal, since (I - P) T = 0), and kept directions with
//     s_j <= sqrt(eps) s_max get no inverse factors (a pseudo-inverse cutoff);
//   gate contraction theta = G (uL x uR) M and merge M = A B: the adjoints of the
//     linear maps, and the 4 x 4 adjoint of G (uL x uR) for the one-qubit gates.
// The final-state adjoint uses transfer-matrix environments (k_env_axpy,
// k_site_adj2, k_adj_combine); k_rot_grad turns the 2 x 2 adjoints of every layer's
// one-qubit gates into angle derivatives.
#include <float.h>

#include <algorithm>

#include "tnsim_internal.h"

namespace tnsim {

namespace {

template <typename T> struct EpsG;
template <> struct EpsG<float> { static constexpr double v = FLT_EPSILON; };
template <> struct EpsG<double> { static constexpr double v = DBL_EPSILON; };

template <typename C>
__device__ __forceinline__ C cz() { C r; r.x = 0; r.y = 0; return r; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C>
__device__ __forceinline__ void cmac(C& acc, const C& a, const C& b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// Operand of cta_gemm: element (i, j) = p[i * rs + j * cs], conjugated if conj.
template <typename C>
struct Op {
    const C* p;
    int64_t rs, cs;
    bool conj;
    __device__ __forceinline__ C at(int i, int j) const {
        C v = p[(int64_t)i * rs + (int64_t)j * cs];
        if (conj) v.y = -v.y;
        return v;
    }
};

constexpr int GT = 64, GK = 16;

// out(i, j) = alpha * sum_k a(i, k) b(k, j) (+ out(i, j) when acc), for i < M, j < N;
// out element (i, j) at o[i * ors + j * ocs].  Whole CTA (256 threads), 64 x 64 tiles.
template <typename T, typename C>
__device__ void cta_gemm(int M, int N, int K, Op<C> a, Op<C> b, C* o, int64_t ors, int64_t ocs, T alpha, bool acc,
                         C (*As)[GT + 1], C (*Bs)[GT]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int tm = (M + GT - 1) / GT, tn = (N + GT - 1) / GT;
    for (int tile = 0; tile < tm * tn; ++tile) {
        const int m0 = (tile / tn) * GT, n0 = (tile % tn) * GT;
        C r[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) r[i][j] = cz<C>();
        for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = tid + 256 * t;
                const int ii = e / GK, kk = e % GK;          // a: 64 rows x 16
                As[kk][ii] = (m0 + ii < M && k0 + kk < K) ? a.at(m0 + ii, k0 + kk) : cz<C>();
                const int kb = e / GT, jj = e % GT;          // b: 16 x 64 columns
                Bs[kb][jj] = (k0 + kb < K && n0 + jj < N) ? b.at(k0 + kb, n0 + jj) : cz<C>();
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < GK; ++kk) {
                C av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) cmac(r[i][j], av[i], bv[j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ii = m0 + ty + 16 * i;
            if (ii >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int jj = n0 + tx + 16 * j;
                if (jj >= N) continue;
                C* dst = o + (int64_t)ii * ors + (int64_t)jj * ocs;
                C v;
                v.x = alpha * r[i][j].x;
                v.y = alpha * r[i][j].y;
                if (acc) { v.x += dst->x; v.y += dst->y; }
                *dst = v;
            }
        }
    }
    __syncthreads();
}

// block-wide sum of n doubles per thread (n <= 32); result in out[] of every thread
template <int NV>
__device__ void block_sum(double (&v)[NV], double* red /* NV * 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    __syncthreads();
    if (lane == 0)
        for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
    __syncthreads();
    for (int i = 0; i < NV; ++i) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[i * 32 + w];
        v[i] = t;
    }
    __syncthreads();
}

// The backward of one two-qubit update (one CTA of 256 threads per gate).
template <typename T>
__global__ void __launch_bounds__(256) k_gate_bwd(const GradGateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GradGateDesc& d = gd[blockIdx.x];
    __shared__ C As[GK][GT + 1];
    __shared__ C Bs[GK][GT];
    __shared__ double red[32 * 32];
    __shared__ C Gt[16];
    __shared__ double s_sc[4];
    const int chiL = d.chiL, chiM = d.chiM, chiR = d.chiR, k = d.k;
    const int m = 2 * chiL, n = 2 * chiR;
    const int tid = threadIdx.x, nt = blockDim.x;
    const C* Tm = (const C*)d.theta0;        // column-major m x n
    const C* W = (const C*)d.W;              // column-major m x n
    const C* U = (const C*)d.u_post;         // m x k row-major
    const C* cY = (const C*)d.y_post;        // k x n row-major
    const C* Ub = (const C*)d.ub_post;       // m x k
    const C* Bb = (const C*)d.bb_post;       // k x n
    const C* Apre = (const C*)d.a_pre;       // (chiL, 2, chiM) = m x chiM row-major
    const C* Bpre = (const C*)d.b_pre;       // (chiM, 2, chiR) = chiM x n row-major
    // scratch: nine regions of cm^2 elements (cm = 2 chi_cap >= m, n, k), whatever shapes
    // they hold (X1 is m x k in the null-space term, dd x k in the discarded one)
    C* S = (C*)d.scratch;
    const size_t R = (size_t)d.cm * d.cm;
    C* Tb = S;                               // m x n row-major
    C* Yb = S + R;                           // k x n
    C* Ut = S + 2 * R;                       // m x k
    C* Ua = S + 3 * R;                       // m x nz column-major (nonzero left singular vectors)
    C* Q1 = S + 4 * R;                       // nz x k
    C* X1 = S + 5 * R;                       // m x k or dd x k
    C* X2 = S + 6 * R;                       // k x n or dd x n
    C* Mm = S + 7 * R;                       // m x n (merge)
    C* Mb = S + 8 * R;                       // m x n, or k x n

    // scalars: k, norms, nonzero count, renormalisation
    if (tid == 0) {
        double f2 = 0.0, k2 = 0.0;
        for (int j = 0; j < n; ++j) f2 += d.s2[j];
        for (int j = 0; j < k; ++j) k2 += d.s2[j];
        const double thr = EpsG<T>::v * (double)max(m, n);
        int nz = 0;
        const double smax2 = d.s2[0];
        for (int j = 0; j < min(m, n); ++j)
            if (d.s2[j] > thr * thr * smax2) nz = j + 1;
        if (nz < k) nz = k;
        s_sc[0] = f2;
        s_sc[1] = k2;
        s_sc[2] = (double)nz;
        s_sc[3] = (d.renorm && k2 > 0.0) ? sqrt(f2 / k2) : 1.0;
    }
    __syncthreads();
    const double F2 = s_sc[0], K2 = s_sc[1], c = s_sc[3];
    const int nz = (int)s_sc[2];
    // dc = 2 Re <Bb, Y>, Y = cY / c
    double dl[1] = {0.0};
    for (int i = tid; i < k * n; i += nt) {
        const C b = Bb[i], y = cY[i];
        dl[0] += (double)b.x * y.x + (double)b.y * y.y;
    }
    block_sum<1>(dl, red);
    const double dldc = 2.0 * dl[0] / c;
    const bool ren = d.renorm && K2 > 0.0;
    // Yb = c Bb - (dc c / 2K2) Y
    {
        const T a1 = (T)c, a2 = ren ? (T)(-dldc * c / (2.0 * K2) / c) : (T)0;
        for (int i = tid; i < k * n; i += nt) {
            const C b = Bb[i], y = cY[i];
            C v;
            v.x = a1 * b.x + a2 * y.x;
            v.y = a1 * b.y + a2 * y.y;
            Yb[i] = v;
        }
    }
    __syncthreads();
    // Tb = U Yb + (dc c / 2F2) T
    cta_gemm<T, C>(m, n, k, Op<C>{U, k, 1, false}, Op<C>{Yb, n, 1, false}, Tb, n, 1, (T)1, false, As, Bs);
    if (ren) {
        const T a3 = (T)(dldc * c / (2.0 * F2));
        for (int i = tid; i < m * n; i += nt) {
            const int row = i / n, col = i % n;
            const C t = Tm[(size_t)col * m + row];
            Tb[i].x += a3 * t.x;
            Tb[i].y += a3 * t.y;
        }
        __syncthreads();
    }
    // Ut = Ub + T Yb^H
    for (int i = tid; i < m * k; i += nt) Ut[i] = Ub[i];
    __syncthreads();
    cta_gemm<T, C>(m, k, n, Op<C>{Tm, 1, m, false}, Op<C>{Yb, 1, n, true}, Ut, k, 1, (T)1, true, As, Bs);
    const bool need_null = nz < m, need_disc = nz > k;
    if (need_null || need_disc) {
        // Ua[:, j] = W[:, perm[j]] / s_j for j < nz (column-major m x nz)
        for (int i = tid; i < m * nz; i += nt) {
            const int j = i / m, row = i % m;
            const double s2j = d.s2[j];
            const T f = s2j > 0.0 ? (T)(1.0 / sqrt(s2j)) : (T)0;
            C w = W[(size_t)d.perm[j] * m + row];
            w.x *= f;
            w.y *= f;
            Ua[i] = w;
        }
        __syncthreads();
        // Q1 = Ua^H Ut (nz x k)
        cta_gemm<T, C>(nz, k, m, Op<C>{Ua, m, 1, true}, Op<C>{Ut, k, 1, false}, Q1, k, 1, (T)1, false, As, Bs);
    }
    // directions below tau s_max get no inverse factors (pseudo-inverse cutoff, tau = sqrt(eps))
    const double tau2s = EpsG<T>::v * d.s2[0];
    if (need_null) {
        // (I - P) Ut = (I - P) Ub exactly ((I - P) T = 0); X1 = Ub - Ua (Ua^H Ub), then
        // Tb += X1 S_k^-2 Y.  Mb holds Ua^H Ub (nz x k) meanwhile.
        cta_gemm<T, C>(nz, k, m, Op<C>{Ua, m, 1, true}, Op<C>{Ub, k, 1, false}, Mb, k, 1, (T)1, false, As, Bs);
        for (int i = tid; i < m * k; i += nt) X1[i] = Ub[i];
        __syncthreads();
        cta_gemm<T, C>(m, k, nz, Op<C>{Ua, 1, m, false}, Op<C>{Mb, k, 1, false}, X1, k, 1, (T)-1, true, As, Bs);
        // X2 = S_k^-2 Y (k x n), Y = cY / c
        for (int i = tid; i < k * n; i += nt) {
            const int j = i / n;
            const T f = d.s2[j] > tau2s ? (T)(1.0 / (c * d.s2[j])) : (T)0;
            C y = cY[i];
            y.x *= f;
            y.y *= f;
            X2[i] = y;
        }
        __syncthreads();
        cta_gemm<T, C>(m, n, k, Op<C>{X1, k, 1, false}, Op<C>{X2, n, 1, false}, Tb, n, 1, (T)1, true, As, Bs);
    }
    if (need_disc) {
        const int dd = nz - k;
        // Lorentzian broadening of the cut's denominators on the scale of their rounding
        // error: s_j^2 - s_l^2 carries an absolute error ~ eps s_max (s_j + s_l), so the
        // broadening is (eps s_max (s_j + s_l))^2 -- it regularises unresolved (degenerate)
        // pairs, where the truncated map is not differentiable, and leaves small but
        // separated singular values alone
        const double e2s = EpsG<T>::v * EpsG<T>::v * d.s2[0];
        // X1 = G o B_D (dd x k), B_D = rows k.. of Q1
        for (int i = tid; i < dd * k; i += nt) {
            const int l = i / k, j = i % k;
            const double dj = d.s2[j] - d.s2[k + l];
            const double sum = sqrt(d.s2[j]) + sqrt(fmax(d.s2[k + l], 0.0));
            const double eps_b = e2s * sum * sum;
            const T g = d.s2[j] > tau2s ? (T)(dj / (dj * dj + eps_b)) : (T)0;
            C b = Q1[(size_t)(k + l) * k + j];
            b.x *= g;
            b.y *= g;
            X1[i] = b;
        }
        __syncthreads();
        // Z T = U_D (Gb Y): X2 = Gb Y (dd x n), Tb += Ua_D X2
        cta_gemm<T, C>(dd, n, k, Op<C>{X1, k, 1, false}, Op<C>{cY, n, 1, false}, X2, n, 1, (T)(1.0 / c), false, As, Bs);
        cta_gemm<T, C>(m, n, dd, Op<C>{Ua + (size_t)k * m, 1, m, false}, Op<C>{X2, n, 1, false}, Tb, n, 1, (T)1, true,
                       As, Bs);
        // Z^H T = U Gb^H (U_D^H T): X2 = U_D^H T (dd x n), Mb (scratch) = Gb^H X2 (k x n), Tb += U Mb
        cta_gemm<T, C>(dd, n, m, Op<C>{Ua + (size_t)k * m, m, 1, true}, Op<C>{Tm, 1, m, false}, X2, n, 1, (T)1, false,
                       As, Bs);
        cta_gemm<T, C>(k, n, dd, Op<C>{X1, 1, k, true}, Op<C>{X2, n, 1, false}, Mb, n, 1, (T)1, false, As, Bs);
        cta_gemm<T, C>(m, n, k, Op<C>{U, k, 1, false}, Op<C>{Mb, n, 1, false}, Tb, n, 1, (T)1, true, As, Bs);
    }
    // effective gate G (uL x uR) in shared memory
    if (tid < 16) {
        const int o = tid >> 2, i = tid & 3;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 4; ++j) {
            const double gr = d.g4[2 * (o * 4 + j)], gi = d.g4[2 * (o * 4 + j) + 1];
            double ar = ((j >> 1) == (i >> 1)) ? 1.0 : 0.0, ai = 0.0;
            double br = ((j & 1) == (i & 1)) ? 1.0 : 0.0, bi = 0.0;
            if (d.uL) { ar = d.uL[2 * ((j >> 1) * 2 + (i >> 1))]; ai = d.uL[2 * ((j >> 1) * 2 + (i >> 1)) + 1]; }
            if (d.uR) { br = d.uR[2 * ((j & 1) * 2 + (i & 1))]; bi = d.uR[2 * ((j & 1) * 2 + (i & 1)) + 1]; }
            const double kr = ar * br - ai * bi, ki = ar * bi + ai * br;
            re += gr * kr - gi * ki;
            im += gr * ki + gi * kr;
        }
        Gt[tid].x = (T)re;
        Gt[tid].y = (T)im;
    }
    // merge M = A B (m x n row-major)
    cta_gemm<T, C>(m, n, chiM, Op<C>{Apre, chiM, 1, false}, Op<C>{Bpre, n, 1, false}, Mm, n, 1, (T)1, false, As, Bs);
    // Mb[(l,c),(d,r)] = sum_ab conj(Gt[2a+b][2c+d]) Tb[(l,a),(b,r)]; Gtb = sum_{l,r} Tb conj(M)
    double gacc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) gacc[i] = 0.0;
    for (int i = tid; i < chiL * chiR; i += nt) {
        const int l = i / chiR, r = i % chiR;
        C tb[4], mm[4];
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            tb[ab] = Tb[(size_t)(2 * l + (ab >> 1)) * n + (ab & 1) * chiR + r];
            mm[ab] = Mm[(size_t)(2 * l + (ab >> 1)) * n + (ab & 1) * chiR + r];
        }
#pragma unroll
        for (int cd = 0; cd < 4; ++cd) {
            C acc = cz<C>();
#pragma unroll
            for (int ab = 0; ab < 4; ++ab) cmac(acc, cconj(Gt[ab * 4 + cd]), tb[ab]);
            Mb[(size_t)(2 * l + (cd >> 1)) * n + (cd & 1) * chiR + r] = acc;
        }
#pragma unroll
        for (int ab = 0; ab < 4; ++ab)
#pragma unroll
            for (int cd = 0; cd < 4; ++cd) {
                const C a = tb[ab], b = mm[cd];   // a conj(b)
                gacc[2 * (ab * 4 + cd)] += (double)a.x * b.x + (double)a.y * b.y;
                gacc[2 * (ab * 4 + cd) + 1] += (double)a.y * b.x - (double)a.x * b.y;
            }
    }
    block_sum<32>(gacc, red);
    __syncthreads();
    // site adjoints: Ab = Mb B^H (m x chiM), Bb = A^H Mb (chiM x n)
    cta_gemm<T, C>(m, chiM, n, Op<C>{Mb, n, 1, false}, Op<C>{Bpre, 1, n, true}, (C*)d.ab_pre, chiM, 1, (T)1, false,
                   As, Bs);
    cta_gemm<T, C>(chiM, n, m, Op<C>{Apre, 1, chiM, true}, Op<C>{Mb, n, 1, false}, (C*)d.bb_pre, n, 1, (T)1, false,
                   As, Bs);
    // Kb = G^H Gtb; uLb[a,c] = sum_bd Kb[(ab),(cd)] conj(uR[b,d]); uRb[b,d] = sum_ac Kb[...] conj(uL[a,c])
    if (tid == 0) {
        double kb[32];
        for (int rI = 0; rI < 4; ++rI)
            for (int cI = 0; cI < 4; ++cI) {
                double re = 0.0, im = 0.0;
                for (int j = 0; j < 4; ++j) {
                    const double gr = d.g4[2 * (j * 4 + rI)], gi = -d.g4[2 * (j * 4 + rI) + 1];   // conj(G[j][rI])
                    const double xr = gacc[2 * (j * 4 + cI)], xi = gacc[2 * (j * 4 + cI) + 1];
                    re += gr * xr - gi * xi;
                    im += gr * xi + gi * xr;
                }
                kb[2 * (rI * 4 + cI)] = re;
                kb[2 * (rI * 4 + cI) + 1] = im;
            }
        auto u_at = [](const double* u, int r, int cc, double& ur, double& ui) {
            if (u) { ur = u[2 * (r * 2 + cc)]; ui = u[2 * (r * 2 + cc) + 1]; }
            else { ur = (r == cc) ? 1.0 : 0.0; ui = 0.0; }
        };
        for (int a = 0; a < 2; ++a)
            for (int cc = 0; cc < 2; ++cc) {
                double lr = 0.0, li = 0.0, rr = 0.0, ri = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int dd = 0; dd < 2; ++dd) {
                        double vr, vi;
                        // uLb[a][cc] += Kb[(a b),(cc dd)] conj(uR[b][dd])
                        u_at(d.uR, b, dd, vr, vi);
                        const double kr = kb[2 * ((2 * a + b) * 4 + 2 * cc + dd)], ki = kb[2 * ((2 * a + b) * 4 + 2 * cc + dd) + 1];
                        lr += kr * vr + ki * vi;
                        li += ki * vr - kr * vi;
                        // uRb[a][cc] (as [b][d] = [a][cc]) += Kb[(b' a),(d' cc)] conj(uL[b'][d'])
                        u_at(d.uL, b, dd, vr, vi);
                        const double kr2 = kb[2 * ((2 * b + a) * 4 + 2 * dd + cc)], ki2 = kb[2 * ((2 * b + a) * 4 + 2 * dd + cc) + 1];
                        rr += kr2 * vr + ki2 * vi;
                        ri += ki2 * vr - kr2 * vi;
                    }
                d.ubar_l[2 * (a * 2 + cc)] += lr;
                d.ubar_l[2 * (a * 2 + cc) + 1] += li;
                d.ubar_r[2 * (a * 2 + cc)] += rr;
                d.ubar_r[2 * (a * 2 + cc) + 1] += ri;
            }
    }
}

// ---------------------------------------------------------------------------
// final-state adjoint helpers (environments are compact chi x chi, chi read on the device)

template <typename T>
__global__ void k_env_axpy(typename CT<T>::type* __restrict__ dst, const typename CT<T>::type* __restrict__ src,
                           const int* __restrict__ chi, int bond, double coef, int zero_first) {
    const int c = chi[bond];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c * c; i += gridDim.x * blockDim.x) {
        auto v = zero_first ? cz<typename CT<T>::type>() : dst[i];
        if (src) {
            v.x += (T)coef * src[i].x;
            v.y += (T)coef * src[i].y;
        }
        dst[i] = v;
    }
}

// out[l, p, r] += coef sum_{l'} E[l, l'] sum_{p'} O[p, p'] tmp[l', p', r]
// (tmp = A Rt from the right-transfer pass; E: left environment, bra x ket)
template <typename T>
__global__ void k_site_adj2(const typename CT<T>::type* __restrict__ E, const double* __restrict__ op,
                            const typename CT<T>::type* __restrict__ tmp, const int* __restrict__ chi, int q,
                            double coef, typename CT<T>::type* __restrict__ out) {
    using C = typename CT<T>::type;
    const int cl = chi[q], cr = chi[q + 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)cl * 2 * cr) return;
    const int l = (int)(t / (2 * cr)), rem = (int)(t % (2 * cr)), p = rem / cr, r = rem % cr;
    C o0, o1;
    o0.x = (T)op[2 * (p * 2)]; o0.y = (T)op[2 * (p * 2) + 1];
    o1.x = (T)op[2 * (p * 2 + 1)]; o1.y = (T)op[2 * (p * 2 + 1) + 1];
    C acc = cz<C>();
    for (int lp = 0; lp < cl; ++lp) {
        C w = cz<C>();
        cmac(w, o0, tmp[((size_t)lp * 2 + 0) * cr + r]);
        cmac(w, o1, tmp[((size_t)lp * 2 + 1) * cr + r]);
        cmac(acc, E[(size_t)l * cl + lp], w);
    }
    out[t].x += (T)coef * acc.x;
    out[t].y += (T)coef * acc.y;
}

// Ab = (AH - (Hsum / N) AN) / N with Hsum, N the 1 x 1 closing environments (device)
template <typename T>
__global__ void k_adj_combine(typename CT<T>::type* __restrict__ ah, const typename CT<T>::type* __restrict__ an,
                              const typename CT<T>::type* __restrict__ hsum, const typename CT<T>::type* __restrict__ nrm,
                              int64_t count) {
    const double N = nrm->x, E = hsum->x / N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        auto v = ah[i];
        const auto w = an[i];
        v.x = (T)((v.x - E * w.x) / N);
        v.y = (T)((v.y - E * w.y) / N);
        ah[i] = v;
    }
}

// one-qubit gates u = R_{a_last}(t_last) ... R_{a_0}(t_0) of every (layer, qubit) from angles
__device__ void rot_mat(char ax, double t, double* r /* 8 */) {
    const double c = cos(0.5 * t), s = sin(0.5 * t);
    // cos I - i sin P
    for (int i = 0; i < 8; ++i) r[i] = 0.0;
    r[0] = c; r[6] = c;
    if (ax == 'X') { r[3] = -s; r[5] = -s; }
    else if (ax == 'Y') { r[2] = -s; r[4] = s; }
    else { r[1] = -s; r[7] = s; }
}
__device__ void mul22(const double* a, const double* b, double* o) {
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 2; ++k) {
                const double ar = a[2 * (2 * i + k)], ai = a[2 * (2 * i + k) + 1];
                const double br = b[2 * (2 * k + j)], bi = b[2 * (2 * k + j) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            o[2 * (2 * i + j)] = re;
            o[2 * (2 * i + j) + 1] = im;
        }
}

__global__ void k_rot_build(const RotLayer* __restrict__ rl, int n_layers, int n, double* __restrict__ u1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_layers * n) return;
    const int L = i / n, q = i % n;
    const RotLayer& R = rl[L];
    if (R.n_rot == 0) return;
    double u[8] = {1, 0, 0, 0, 0, 0, 1, 0}, r[8], t[8];
    for (int j = 0; j < R.n_rot; ++j) {
        rot_mat(R.axes[j], R.theta[(size_t)q * R.n_rot + j], r);
        mul22(r, u, t);
        for (int e = 0; e < 8; ++e) u[e] = t[e];
    }
    for (int e = 0; e < 8; ++e) u1[R.u1_off + (size_t)q * 8 + e] = u[e];
}

// dE/dt_j = 2 Re <ub, du/dt_j>, dR_a/dt = (-i/2) P_a R_a
__global__ void k_rot_grad(const RotLayer* __restrict__ rl, int n_layers, int n, const double* __restrict__ ub,
                           double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_layers * n) return;
    const int L = i / n, q = i % n;
    const RotLayer& R = rl[L];
    const double* b = ub + R.u1_off + (size_t)q * 8;
    for (int j = 0; j < R.n_rot; ++j) {
        double u[8] = {1, 0, 0, 0, 0, 0, 1, 0}, r[8], t[8];
        for (int jj = 0; jj < R.n_rot; ++jj) {
            rot_mat(R.axes[jj], R.theta[(size_t)q * R.n_rot + jj], r);
            if (jj == j) {
                // (-i/2) P r
                double p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                const char ax = R.axes[jj];
                if (ax == 'X') { p[0 + 2] = 1; p[4] = 1; }
                else if (ax == 'Y') { p[3] = -1; p[5] = 1; }
                else { p[0] = 1; p[6] = -1; }
                double pr[8];
                mul22(p, r, pr);
                for (int e = 0; e < 4; ++e) {
                    const double re = pr[2 * e], im = pr[2 * e + 1];
                    r[2 * e] = 0.5 * im;       // (-i/2)(re + i im) = im/2 - i re/2
                    r[2 * e + 1] = -0.5 * re;
                }
            }
            mul22(r, u, t);
            for (int e = 0; e < 8; ++e) u[e] = t[e];
        }
        double acc = 0.0;
        for (int e = 0; e < 4; ++e) acc += b[2 * e] * u[2 * e] + b[2 * e + 1] * u[2 * e + 1];
        grad[R.grad_off + (size_t)q * R.n_rot + j] = 2.0 * acc;
    }
}

// unpaired site of a layer with one-qubit gate u: Ab_pre[l,s,r] = sum_p conj(u[p,s]) Ab[l,p,r],
// ub[p,s] += sum_{l,r} Ab[l,p,r] conj(A_pre[l,s,r]); one CTA per site
template <typename T>
__global__ void __launch_bounds__(256) k_site1_bwd(const Site1Bwd* __restrict__ sd) {
    using C = typename CT<T>::type;
    const Site1Bwd& d = sd[blockIdx.x];
    const C* ab = (const C*)d.ab_post;
    const C* a = (const C*)d.a_pre;
    C* out = (C*)d.ab_pre;
    const int cl = d.cl, cr = d.cr;
    double u[8];
    for (int e = 0; e < 8; ++e) u[e] = d.u[e];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < cl * cr; i += blockDim.x) {
        const int l = i / cr, r = i % cr;
        const C b0 = ab[((size_t)l * 2 + 0) * cr + r], b1 = ab[((size_t)l * 2 + 1) * cr + r];
        const C a0 = a[((size_t)l * 2 + 0) * cr + r], a1 = a[((size_t)l * 2 + 1) * cr + r];
        const C bb[2] = {b0, b1}, aa[2] = {a0, a1};
        for (int s = 0; s < 2; ++s) {
            // sum_p conj(u[p][s]) bb[p]
            double re = 0.0, im = 0.0;
            for (int p = 0; p < 2; ++p) {
                const double ur = u[2 * (p * 2 + s)], ui = -u[2 * (p * 2 + s) + 1];
                re += ur * bb[p].x - ui * bb[p].y;
                im += ur * bb[p].y + ui * bb[p].x;
            }
            C v;
            v.x = (T)re;
            v.y = (T)im;
            out[((size_t)l * 2 + s) * cr + r] = v;
        }
        for (int p = 0; p < 2; ++p)
            for (int s = 0; s < 2; ++s) {
                acc[2 * (p * 2 + s)] += (double)bb[p].x * aa[s].x + (double)bb[p].y * aa[s].y;
                acc[2 * (p * 2 + s) + 1] += (double)bb[p].y * aa[s].x - (double)bb[p].x * aa[s].y;
            }
    }
    __shared__ double red[8 * 32];
    block_sum<8>(acc, red);
    if (threadIdx.x == 0)
        for (int e = 0; e < 8; ++e) d.ubar[e] += acc[e];
}

}  // namespace

template <typename T>
cudaError_t launch_gate_bwd(const GradGateDesc* d, int n_gates, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    k_gate_bwd<T><<<n_gates, 256, 0, s>>>(d);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_site1_bwd(const Site1Bwd* d, int n_sites, cudaStream_t s) {
    if (n_sites <= 0) return cudaSuccess;
    k_site1_bwd<T><<<n_sites, 256, 0, s>>>(d);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_env_axpy(void* dst, const void* src, const int* chi, int bond, double coef, int zero_first,
                            int chi_cap, cudaStream_t s) {
    using C = typename CT<T>::type;
    const int blocks = (chi_cap * chi_cap + 255) / 256;
    k_env_axpy<T><<<blocks > 0 ? blocks : 1, 256, 0, s>>>((C*)dst, (const C*)src, chi, bond, coef, zero_first);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_site_adj2(const void* E, const double* op, const void* tmp, const int* chi, int q, double coef,
                             void* out, int chi_cap, cudaStream_t s) {
    using C = typename CT<T>::type;
    const int64_t tot = (int64_t)chi_cap * 2 * chi_cap;
    k_site_adj2<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const C*)E, op, (const C*)tmp, chi, q, coef, (C*)out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_adj_combine(void* ah, const void* an, const void* hsum, const void* nrm, int64_t count,
                               cudaStream_t s) {
    using C = typename CT<T>::type;
    k_adj_combine<T><<<(unsigned)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, s>>>(
        (C*)ah, (const C*)an, (const C*)hsum, (const C*)nrm, count);
    return cudaGetLastError();
}
cudaError_t launch_rot_build(const RotLayer* rl, int n_layers, int n, double* u1, cudaStream_t s) {
    const int tot = n_layers * n;
    k_rot_build<<<(tot + 127) / 128, 128, 0, s>>>(rl, n_layers, n, u1);
    return cudaGetLastError();
}
cudaError_t launch_rot_grad(const RotLayer* rl, int n_layers, int n, const double* ub, double* grad, cudaStream_t s) {
    const int tot = n_layers * n;
    k_rot_grad<<<(tot + 127) / 128, 128, 0, s>>>(rl, n_layers, n, ub, grad);
    return cudaGetLastError();
}

#define TNSIM_GRAD_INST(T)                                                                                      \
    template cudaError_t launch_gate_bwd<T>(const GradGateDesc*, int, cudaStream_t);                              \
    template cudaError_t launch_site1_bwd<T>(const Site1Bwd*, int, cudaStream_t);                                 \
    template cudaError_t launch_env_axpy<T>(void*, const void*, const int*, int, double, int, int, cudaStream_t); \
    template cudaError_t launch_site_adj2<T>(const void*, const double*, const void*, const int*, int, double,   \
                                             void*, int, cudaStream_t);                                           \
    template cudaError_t launch_adj_combine<T>(void*, const void*, const void*, const void*, int64_t, cudaStream_t);
TNSIM_GRAD_INST(float)
TNSIM_GRAD_INST(double)
#undef TNSIM_GRAD_INST

}  // namespace tnsim
