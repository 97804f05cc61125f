// Two-qubit update in canonical (Hastings) form.
//
// The state is kept right-canonical, with the singular values Lam_b of every bond
// stored beside it (Hastings, "Light-cone matrix product", J. Math. Phys. 50 (2009)).
// For the pair (q, q+1) with theta = G (A_q A_{q+1}) as in the paper's update:
//   * the SVD operand is diag(Lam_q) theta: rows (l, a) scaled by Lam_q[l], so its
//     singular values are the Schmidt coefficients of cut q+1 and the truncation
//     acts on them (k_scale_rows, before the Jacobi SVD);
//   * the right site becomes V^H: row j = u_j^H diag(Lam_q) theta / s_j, formed by
//     k_right from the Jacobi columns w_j = u_j s_j, then re-orthonormalised
//     (k_orth_rows).  Row j of that product carries an error of about eps s_max / s_j
//     (the Jacobi's backward error divided by s_j), mostly along the rows of larger
//     singular values; modified Gram-Schmidt in the order of decreasing s removes
//     exactly those components, and what it leaves (along rows of smaller s) enters
//     the state weighted by those smaller singular values;
//   * the left site becomes theta V (times the renormalisation factor), with no
//     division by Lam_q (k_left_canon, after k_right).
// Bond q+1 then stores the kept (renormalised) singular values, as in the paper's form.
#include "tnsim_internal.h"

namespace tnsim {

namespace {

template <typename C>
__device__ __forceinline__ void cfma_conj_b(C& acc, const C& a, const C& b) {   // acc += a conj(b)
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}

// W[(l,a), c] *= Lam_q[l] (column-major, m = 2 chi_L rows) and out->frob2 = |W|_F^2
// (FP64), one CTA per gate; gates in the paper's form are left alone.
template <typename T>
__global__ void __launch_bounds__(512) k_scale_rows(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.x];
    if (!d.canon) return;
    const int q = d.q;
    const int m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    const int lk = *d.lam_k;
    C* Wm = (C*)d.W;
    double acc = 0.0;
    const int64_t total = (int64_t)m * n;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int l = (int)(i % m) >> 1;
        const T f = (l < lk) ? (T)d.lam[l] : (T)1;
        C v = Wm[i];
        v.x *= f;
        v.y *= f;
        Wm[i] = v;
        acc = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, acc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[16];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        d.out->frob2 = t;
    }
}

// Modified Gram-Schmidt of the k rows (length n) of the new right site, in the
// order of decreasing singular value (the stored row order); one CTA per gate.
template <typename T>
__global__ void __launch_bounds__(1024) k_orth_rows(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.x];
    if (!d.canon) return;
    const int n = 2 * d.chi[d.q + 2];
    const int k = d.out->k;
    C* R = (C*)d.siteB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ T s_inv;
    for (int j = 0; j < k; ++j) {
        C* rj = R + (size_t)j * n;
        if (warp == 0) {
            T a = 0;
            for (int c = lane; c < n; c += 32) a = fma(rj[c].x, rj[c].x, fma(rj[c].y, rj[c].y, a));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) s_inv = a > (T)0 ? (T)1 / sqrt(a) : (T)0;
        }
        __syncthreads();
        const T f = s_inv;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            rj[c].x *= f;
            rj[c].y *= f;
        }
        __syncthreads();
        // rows i > j lose their component along row j: r_i -= (r_j^H r_i) r_j
        for (int i = j + 1 + warp; i < k; i += nw) {
            C* ri = R + (size_t)i * n;
            T pr = 0, pi = 0;
            for (int c = lane; c < n; c += 32) {
                const C a = rj[c], b = ri[c];
                pr = fma(a.x, b.x, fma(a.y, b.y, pr));
                pi = fma(a.x, b.y, fma(-a.y, b.x, pi));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                pr += __shfl_xor_sync(0xffffffffu, pr, o);
                pi += __shfl_xor_sync(0xffffffffu, pi, o);
            }
            for (int c = lane; c < n; c += 32) {
                const C a = rj[c];
                C b = ri[c];
                b.x -= pr * a.x - pi * a.y;
                b.y -= pr * a.y + pi * a.x;
                ri[c] = b;
            }
        }
        __syncthreads();
    }
}

constexpr int LC_M = 64, LC_J = 64, LC_K = 16;

// left site A'[(l,a), j] = scale * sum_c theta0[(l,a), c] conj(B'[j, c]), with theta0
// column-major (m x n) and B' the new right site (k x n, row-major); 64 x 64 tile per CTA
template <typename T>
__global__ void __launch_bounds__(256) k_left_canon(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.z];
    if (!d.canon) return;
    const int q = d.q;
    const int m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    const int k = d.out->k;
    const int r0 = blockIdx.x * LC_M, j0 = blockIdx.y * LC_J;
    if (r0 >= m || j0 >= k) return;
    __shared__ C As[LC_K][LC_M];
    __shared__ C Bs[LC_K][LC_J + 1];
    const C* T0 = (const C*)d.theta0;
    const C* Bp = (const C*)d.siteB;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j].x = 0; acc[i][j].y = 0; }
    for (int c0 = 0; c0 < n; c0 += LC_K) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t;
            // theta0 tile: LC_K columns x LC_M rows, rows fastest (coalesced)
            const int cc = e / LC_M, rr = e % LC_M;
            C a; a.x = 0; a.y = 0;
            if (c0 + cc < n && r0 + rr < m) a = T0[(size_t)(c0 + cc) * m + r0 + rr];
            As[cc][rr] = a;
            // B' tile: LC_J rows (j) x LC_K columns (c), columns fastest
            const int jj = e / LC_K, kc = e % LC_K;
            C b; b.x = 0; b.y = 0;
            if (j0 + jj < k && c0 + kc < n) b = Bp[(size_t)(j0 + jj) * n + c0 + kc];
            Bs[kc][jj] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < LC_K; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma_conj_b(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    const T sc = (T)d.out->scale;
    C* Ap = (C*)d.siteA;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx + 16 * j;
            if (jj < k) {
                C v; v.x = acc[i][j].x * sc; v.y = acc[i][j].y * sc;
                Ap[(size_t)r * k + jj] = v;
            }
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_scale_rows(const GateDesc* d, int n_gates, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    k_scale_rows<T><<<n_gates, 512, 0, s>>>(d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_left_canon(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    k_orth_rows<T><<<n_gates, 1024, 0, s>>>(d);
    dim3 grid((m_max + LC_M - 1) / LC_M, (k_max + LC_J - 1) / LC_J, n_gates);
    k_left_canon<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t launch_scale_rows<float>(const GateDesc*, int, cudaStream_t);
template cudaError_t launch_scale_rows<double>(const GateDesc*, int, cudaStream_t);
template cudaError_t launch_left_canon<float>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_left_canon<double>(const GateDesc*, int, int, int, cudaStream_t);

}  // namespace tnsim
