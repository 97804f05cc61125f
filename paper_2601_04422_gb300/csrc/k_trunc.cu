// Truncation and absorption of the two-qubit update, and the one-qubit update.
//
//  k_colnorm2 : squared column norms of the converged W (the squared singular
//               values), FP64 accumulation, 32 columns per CTA over all gates.
//  k_truncate : one CTA per gate.  A bitonic sort orders the squared norms
//               descending (ties: lower column first); the kept rank is
//                 k = max(1, min(chi_max, #{s_j > eps*max(m,n)*s_max},
//                                smallest k with sum_{j>=k} s_j^2 <= cutoff*sum s_j^2))
//               (Sec. II.A: truncate the bond; Sec. IV.A: "the bond dimension can be
//               truncated").  The discarded weight and the renormalisation factor
//               sqrt(sum s^2 / sum_{j<k} s^2) are FP64.  Writes chi[q+1] = k.
//  k_left     : new left site = left singular vectors (Sec. III.A "Two Qubit Gate"):
//               A'[(l,p0), j] = W[(l,p0), perm_j] / s_{perm_j}, a gather + transpose
//               through a shared-memory tile (coalesced reads and writes).
//  k_site1q   : A'[l,p',r] = sum_p U[p',p] A[l,p,r]  (Eq. 3), in place.
#include <float.h>

#include "tnsim_internal.h"

namespace tnsim {

template <typename T> struct EpsT;
template <> struct EpsT<float> { static constexpr double v = FLT_EPSILON; };
template <> struct EpsT<double> { static constexpr double v = DBL_EPSILON; };

constexpr int TR_THREADS = 512;
constexpr int TR_MAXN = 1024;
constexpr int CN_COLS = 32;        // columns per CTA of k_colnorm2 (8 warps, 4 columns each)

// a comes after b in the sorted order (descending value, ascending index)
__device__ __forceinline__ bool after(double ka, int ia, double kb, int ib) {
    return ka < kb || (ka == kb && ia > ib);
}

// Squared column norms of the converged W, spread over many CTAs: grid (column chunks
// of 32, gates), one warp per column at a time, 16-byte loads, per-lane SqAcc sums
// (double-length FP32 for complex64), then an FP64 warp reduction.  The unsorted
// values go to d.s2 (k_truncate sorts them in place).
template <typename T>
__global__ void __launch_bounds__(256) k_colnorm2(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.y];
    const int q = d.q;
    const int m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    const int c0 = blockIdx.x * CN_COLS;
    if (c0 >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // m is even: a column is m / 2 (complex64) or m (complex128) 16-byte units
    constexpr int PER = 16 / (int)sizeof(C);      // complex elements per 16-byte unit
    const int units = m / PER;
    for (int col = c0 + warp; col < min(c0 + CN_COLS, n); col += 8) {
        const C* wc = (const C*)d.W + (size_t)col * m;
        SqAcc<T> sq;
        for (int u = lane; u < units; u += 32) {
            if constexpr (sizeof(C) == 8) {
                const float4 v = __ldcg(reinterpret_cast<const float4*>(wc) + u);
                sq.add(v.x);
                sq.add(v.y);
                sq.add(v.z);
                sq.add(v.w);
            } else {
                const double2 z = __ldcg(reinterpret_cast<const double2*>(wc) + u);
                sq.add(z.x);
                sq.add(z.y);
            }
        }
        double acc = sq.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) d.s2[col] = acc;
    }
}

// block-wide sum of one double per thread (TR_THREADS threads); every thread gets it
__device__ __forceinline__ double tr_block_sum(double v, double* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll 1
    for (int w = 0; w < TR_THREADS / 32; ++w) t += red[w];
    return t;
}

// Sort the squared norms, pick the kept rank, discarded weight and renormalisation.
// One CTA per gate: bitonic sort (descending value, then ascending column), then
// parallel reductions and a suffix scan of the sorted values for the cutoff rule.
template <typename T>
__global__ void __launch_bounds__(TR_THREADS) k_truncate(const GateDesc* __restrict__ gd) {
    const GateDesc& d = gd[blockIdx.x];
    const int q = d.q;
    const int chiL = d.chi[q], chiM = d.chi[q + 1], chiR = d.chi[q + 2];
    const int m = 2 * chiL, n = 2 * chiR;
    GateOut* out = d.out;

    __shared__ double key[TR_MAXN];
    __shared__ int idx[TR_MAXN];
    __shared__ double red[TR_THREADS / 32];
    __shared__ double wsum[TR_THREADS / 32];
    __shared__ int s_k;
    __shared__ double s_scale;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int P2 = 1;
    while (P2 < n) P2 <<= 1;

    for (int i = tid; i < P2; i += TR_THREADS) {
        if (i < n) {
            key[i] = __ldcg(d.s2 + i);
            idx[i] = i;
        } else {
            key[i] = -1.0;
            idx[i] = 0x7fffffff;
        }
    }
    __syncthreads();

    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P2; i += TR_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double ka = key[i], kb = key[ixj];
                    const int ia = idx[i], ib = idx[ixj];
                    const bool up = (i & kk) == 0;
                    const bool sw = up ? after(ka, ia, kb, ib) : after(kb, ib, ka, ia);
                    if (sw) { key[i] = kb; key[ixj] = ka; idx[i] = ib; idx[ixj] = ia; }
                }
            }
            __syncthreads();
        }
    }

    // each thread owns up to two consecutive sorted entries: 2 tid, 2 tid + 1
    const int j0 = 2 * tid, j1 = 2 * tid + 1;
    const double v0 = j0 < n ? key[j0] : 0.0, v1 = j1 < n ? key[j1] : 0.0;
    const double total = tr_block_sum(v0 + v1, red);
    int k = 1;
    double eps = 0.0, scale = 1.0;
    if (total > 0.0) {
        const double smax = sqrt(key[0]);
        const double thr = EpsT<T>::v * (double)max(m, n) * smax;
        // the values are sorted, so the nonzero ones are a prefix
        const double nzc = tr_block_sum((double)((j0 < n && sqrt(v0) > thr) + (j1 < n && sqrt(v1) > thr)), red);
        const int nonzero = (int)nzc;
        // the rank of an m x n matrix is at most min(m, n); this also bounds the new
        // site shapes by the slot capacities
        k = max(1, min(min(d.chi_max, nonzero), min(m, n)));
        // suffix sums S_j = sum_{i >= j} key[i] (a reverse inclusive scan over the thread
        // pairs): S is non-increasing in j, so the entries with S_j > lim form a prefix
        const double pair = v0 + v1;
        double incl = pair;     // inclusive scan from the last thread down
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_down_sync(0xffffffffu, incl, o);
            if (lane + o < 32) incl += y;
        }
        __syncthreads();
        if (lane == 0) wsum[warp] = incl;      // the warp's total (its lane 0 holds all 32)
        __syncthreads();
        double later = 0.0;                    // the sum of every later warp
        for (int w = warp + 1; w < TR_THREADS / 32; ++w) later += wsum[w];
        const double S0 = incl + later;        // S_{j0}
        const double S1 = S0 - v0;             // S_{j1}
        if (d.cutoff > 0.0) {
            const double lim = d.cutoff * total;
            const double kkc = tr_block_sum((double)((j0 < n && S0 > lim) + (j1 < n && S1 > lim)), red);
            k = max(1, min(k, (int)kkc));
        }
        __syncthreads();
        // discarded and kept weights: S_k and total - S_k
        if (j0 == k && k < n) s_scale = S0;
        if (j1 == k && k < n) s_scale = S1;
        if (tid == 0 && k >= n) s_scale = 0.0;
        __syncthreads();
        const double disc = s_scale, kept = total - disc;
        eps = disc / total;
        if (d.renorm && kept > 0.0) scale = sqrt(total / kept);
        __syncthreads();
    }
    if (tid == 0) {
        s_k = k;
        s_scale = scale;
        out->k = k;
        out->eps = eps;
        out->scale = scale;
        if (d.eps_out) *d.eps_out = eps;
        d.chi[q + 1] = k;
        *d.spec_k = k;
        // a gate whose iteration never ended was abandoned by an idle-timeout (ETIMEOUT)
        if (!out->finished) out->status = 5;
        if (out->status) atomicMax(d.sticky, out->status);
        typedef unsigned long long u64;
        atomicAdd(&d.stats[0], 1ull);
        atomicAdd(&d.stats[1], (u64)out->sweeps);
        atomicAdd(&d.stats[2], out->rotations);
        atomicAdd(&d.stats[3], out->visits);
        atomicAdd(&d.stats[4], out->visits * (u64)m);
        atomicAdd(&d.stats[5], out->rotations * (u64)m);
        atomicAdd(&d.stats[6], (u64)m * (u64)chiM * (u64)n);
        atomicAdd(&d.stats[7], (u64)k * (u64)m * (u64)n);
        if (qr_active(d, m, n)) atomicAdd(&d.stats[8], (u64)2 * (u64)n * (u64)n * (u64)n / 3);
    }
    __syncthreads();
    k = s_k;
    scale = s_scale;
    for (int j = tid; j < n; j += TR_THREADS) {
        d.s2[j] = key[j];
        d.perm[j] = idx[j];
        if (j < k) d.spectrum[j] = sqrt(key[j]) * scale;
    }
}

template <typename T>
cudaError_t launch_truncate(const GateDesc* d, int n_gates, int n_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    dim3 gn((n_max + CN_COLS - 1) / CN_COLS, n_gates, 1);
    k_colnorm2<T><<<gn, 256, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_truncate<T><<<n_gates, TR_THREADS, 0, s>>>(d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_left(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.z];
    if (d.canon) return;   // canonical form: the left site is theta V (k_canon.cu)
    const int q = d.q;
    const int chiL = d.chi[q];
    const int m = 2 * chiL;
    if (qr_active(d, m, 2 * d.chi[q + 2])) return;   // QR-preconditioned: k_left_pre (k_qr.cu)
    const int k = d.out->k;
    const int row0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    if (row0 >= m || j0 >= k) return;
    __shared__ C tile[32][33];
    __shared__ T inv_s[32];
    __shared__ int col_s[32];
    const C* Wm = (const C*)d.W;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (threadIdx.x < 32) {
        // 1 / s_j and the column of each kept j of this tile, once per CTA (FP64 runs at
        // 1/64 of the FP32 rate: not per element)
        const int j = j0 + threadIdx.x;
        const double s2j = j < k ? d.s2[j] : 0.0;
        inv_s[threadIdx.x] = s2j > 0.0 ? (T)(1.0 / sqrt(s2j)) : (T)0;
        col_s[threadIdx.x] = j < k ? d.perm[j] : 0;
    }
    __syncthreads();
    for (int jj = ty; jj < 32; jj += 8) {
        const int j = j0 + jj;
        C v; v.x = 0; v.y = 0;
        if (j < k && row0 + tx < m) {
            const T inv = inv_s[jj];
            v = Wm[(size_t)col_s[jj] * m + row0 + tx];
            v.x *= inv; v.y *= inv;
        }
        tile[jj][tx] = v;
    }
    __syncthreads();
    C* A = (C*)d.siteA;
    for (int rr = ty; rr < 32; rr += 8) {
        const int row = row0 + rr, j = j0 + tx;
        if (row < m && j < k) A[(size_t)row * k + j] = tile[tx][rr];
    }
}

template <typename T>
cudaError_t launch_left(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    dim3 grid((m_max + 31) / 32, (k_max + 31) / 32, n_gates);
    k_left<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_site1q(const Site1Desc* __restrict__ sd) {
    using C = typename CT<T>::type;
    const Site1Desc& s = sd[blockIdx.y];
    const int chiL = s.chi[s.q], chiR = s.chi[s.q + 1];
    C u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { u[i].x = (T)s.u[2 * i]; u[i].y = (T)s.u[2 * i + 1]; }
    C* A = (C*)s.site;
    const int total = chiL * chiR;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int l = t / chiR, r = t - l * chiR;
        C* p0 = A + (size_t)(2 * l) * chiR + r;
        C* p1 = p0 + chiR;
        const C a0 = *p0, a1 = *p1;
        C b0, b1;
        b0.x = u[0].x * a0.x - u[0].y * a0.y + u[1].x * a1.x - u[1].y * a1.y;
        b0.y = u[0].x * a0.y + u[0].y * a0.x + u[1].x * a1.y + u[1].y * a1.x;
        b1.x = u[2].x * a0.x - u[2].y * a0.y + u[3].x * a1.x - u[3].y * a1.y;
        b1.y = u[2].x * a0.y + u[2].y * a0.x + u[3].x * a1.y + u[3].y * a1.x;
        *p0 = b0;
        *p1 = b1;
    }
}

template <typename T>
cudaError_t launch_site1q(const Site1Desc* d, int n_sites, int cap_lr, cudaStream_t s) {
    if (n_sites <= 0) return cudaSuccess;
    int bx = (cap_lr + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, n_sites, 1);
    k_site1q<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t launch_truncate<float>(const GateDesc*, int, int, cudaStream_t);
template cudaError_t launch_truncate<double>(const GateDesc*, int, int, cudaStream_t);
template cudaError_t launch_left<float>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_left<double>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_site1q<float>(const Site1Desc*, int, int, cudaStream_t);
template cudaError_t launch_site1q<double>(const Site1Desc*, int, int, cudaStream_t);

}  // namespace tnsim
