// Perfect sampling of an MPS with memoised prefixes (Sec. III.A "Sampling",
// Sec. IV.A measurement).
//
// Shot s draws qubit q from the weights of its two outcomes given its bits so far:
// with v the (normalised) row vector of its prefix and R_{q+1} the right environment
// of bond q+1,
//     w_b = v A_q[:, b, :],   p_b = w_b R_{q+1} w_b^H,
//     b_q = 1  exactly when  u[s, q] (p0 + p1) >= p0,
// and the prefix becomes w_b / sqrt(p_b) (projection on the outcome, renormalised).
// Using R_{q+1} gives the same weights as first bringing the MPS to right-canonical
// form (where every right environment is the identity).
//
// Memoisation: shots with the same prefix share v, so each site works on the
// distinct prefixes ("nodes") only -- at most min(shots, 2^q) of them -- and a shot
// just carries the index of its node.  Per site:
//   k_cgemm      W = V A_q                 (nodes x 2chi_R)
//   k_cgemm      Y = W' Rt_{q+1}           (2 nodes x chi_R; W' = W as rows (node, b))
//   k_rowdot     p[(node, b)] = Re <w, y>  (FP64 sums)
//   k_decide     every shot: its bit from its uniform, and mark child (node, bit)
//   k_scan       number the marked children: they are the next site's nodes
//   k_project    V'[child] = w_b / sqrt(p_b);  k_advance: every shot moves to its child
// The node count lives in device memory; grids are sized by the host bound
// min(shots, 2^q) and the kernels read the actual count.
#include <algorithm>

#include "tnsim_internal.h"

namespace tnsim {

namespace {

template <typename C>
__device__ __forceinline__ void cmac(C& acc, const C& a, const C& b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

constexpr int GBM = 64, GBN = 64, GBK = 16;

// Cm[M x N] = A[M x K] B[K x N], complex, row-major with leading dimensions;
// M = (*m_dev) * m_mul.  64 x 64 tile per CTA of 256 threads, 4 x 4 outputs each;
// blockIdx.x runs over row tiles (the long side), blockIdx.y over column tiles.
template <typename T>
__global__ void __launch_bounds__(256) k_cgemm(const typename CT<T>::type* __restrict__ A, int lda,
                                               const typename CT<T>::type* __restrict__ B, int ldb,
                                               typename CT<T>::type* __restrict__ Cm, int ldc,
                                               const int* __restrict__ m_dev, int m_mul, int N, int K) {
    using C = typename CT<T>::type;
    const int M = *m_dev * m_mul;
    const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
    if (m0 >= M) return;
    __shared__ C As[GBK][GBM + 1];
    __shared__ C Bs[GBK][GBN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j].x = 0; acc[i][j].y = 0; }
    for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int r = ty + 16 * t, c = tx;          // A tile: row r, column c
            C a; a.x = 0; a.y = 0;
            if (m0 + r < M && k0 + c < K) a = A[(size_t)(m0 + r) * lda + k0 + c];
            As[c][r] = a;
            const int e = tid + 256 * t, rb = e / GBN, cb = e % GBN;   // B tile
            C b; b.x = 0; b.y = 0;
            if (k0 + rb < K && n0 + cb < N) b = B[(size_t)(k0 + rb) * ldb + n0 + cb];
            Bs[rb][cb] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GBK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = m0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx + 16 * j;
            if (c < N) Cm[(size_t)r * ldc + c] = acc[i][j];
        }
    }
}

// p[row] = Re sum_a conj(W[row, a]) Y[row, a] for row < 2 * nodes (FP64 sums); one warp per row
template <typename T>
__global__ void k_rowdot(const typename CT<T>::type* __restrict__ Wr, const typename CT<T>::type* __restrict__ Y,
                         int cr, const int* __restrict__ nodes, double* __restrict__ p) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= 2 * *nodes) return;
    double acc = 0.0;
    for (int a = lane; a < cr; a += 32) {
        const auto w = Wr[(size_t)row * cr + a];
        const auto y = Y[(size_t)row * cr + a];
        acc += (double)w.x * (double)y.x + (double)w.y * (double)y.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) p[row] = acc;
}

// every shot: its bit from its uniform and its node's weights; mark the child
__global__ void k_decide(const double* __restrict__ u, int n, int q, int64_t shots, const int* __restrict__ node_of,
                         const double* __restrict__ p, uint8_t* __restrict__ bits, int* __restrict__ flag) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= shots) return;
    const int i = node_of[s];
    const double p0 = fmax(p[2 * i], 0.0), p1 = fmax(p[2 * i + 1], 0.0);
    const int b = (u[s * n + q] * (p0 + p1) >= p0) ? 1 : 0;
    bits[s * n + q] = (uint8_t)b;
    flag[2 * i + b] = 1;
}

// exclusive scan of the 2 * nodes child flags in one CTA of 1024 threads: child k
// (= 2 node + bit) gets the next site's node index id[k]; parent[id] = k; the new
// node count replaces *nodes and is added to *total
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ flag, int* __restrict__ id,
                                               int* __restrict__ parent, int* __restrict__ nodes,
                                               unsigned long long* __restrict__ total) {
    __shared__ int warp_sum[32];
    __shared__ int s_base;
    const int L = 2 * *nodes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (L + 1023) / 1024;
    const int lo = min(L, tid * per), hi = min(L, lo + per);
    int local = 0;
    for (int k = lo; k < hi; ++k) local += flag[k];
    // block-wide exclusive scan of the per-thread sums
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        warp_sum[lane] = w;   // inclusive over warps
        if (lane == 31) s_base = w;
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? warp_sum[warp - 1] : 0);
    for (int k = lo; k < hi; ++k) {
        if (flag[k]) {
            id[k] = run;
            parent[run] = k;
            ++run;
        } else {
            id[k] = -1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        *nodes = s_base;
        *total += (unsigned long long)s_base;
    }
}

// V'[j, :] = W'[parent[j], :] / sqrt(p[parent[j]]) for j < nodes (the new count)
template <typename T>
__global__ void k_project(const typename CT<T>::type* __restrict__ Wr, const double* __restrict__ p,
                          const int* __restrict__ parent, const int* __restrict__ nodes, int cr,
                          typename CT<T>::type* __restrict__ V) {
    const int j = blockIdx.x;
    if (j >= *nodes) return;
    const int k = parent[j];
    const double pk = p[k];
    const T sc = (T)(pk > 0.0 ? 1.0 / sqrt(pk) : 0.0);
    for (int a = threadIdx.x; a < cr; a += blockDim.x) {
        auto w = Wr[(size_t)k * cr + a];
        w.x *= sc;
        w.y *= sc;
        V[(size_t)j * cr + a] = w;
    }
}

__global__ void k_advance(int64_t shots, int n, int q, const uint8_t* __restrict__ bits, const int* __restrict__ id,
                          int* __restrict__ node_of) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= shots) return;
    node_of[s] = id[2 * node_of[s] + bits[s * n + q]];
}

}  // namespace

template <typename T>
cudaError_t launch_sample_site(const void* site, int cl, int cr, const void* rt_next, int q, int n,
                               int64_t shots, int node_bound, const double* u, uint8_t* bits,
                               SampleWork& w, cudaStream_t s) {
    using C = typename CT<T>::type;
    if (node_bound < 1) node_bound = 1;
    const C* V = (const C*)w.v_cur;
    C* Wm = (C*)w.w;
    C* Y = (C*)w.y;
    // W = V A_q  (nodes x 2cr)
    {
        dim3 g((unsigned)((node_bound + GBM - 1) / GBM), (unsigned)((2 * cr + GBN - 1) / GBN));
        k_cgemm<T><<<g, 256, 0, s>>>(V, cl, (const C*)site, 2 * cr, Wm, 2 * cr, w.nodes, 1, 2 * cr, cl);
    }
    // Y = W' Rt  (2 nodes x cr)
    {
        dim3 g((unsigned)((2 * node_bound + GBM - 1) / GBM), (unsigned)((cr + GBN - 1) / GBN));
        k_cgemm<T><<<g, 256, 0, s>>>(Wm, cr, (const C*)rt_next, cr, Y, cr, w.nodes, 2, cr, cr);
    }
    k_rowdot<T><<<(unsigned)((2 * node_bound + 7) / 8), 256, 0, s>>>(Wm, Y, cr, w.nodes, w.p);
    cudaError_t e = cudaMemsetAsync(w.flag, 0, sizeof(int) * 2 * (size_t)node_bound, s);
    if (e != cudaSuccess) return e;
    const unsigned gs = (unsigned)((shots + 255) / 256);
    k_decide<<<gs, 256, 0, s>>>(u, n, q, shots, w.node_of, w.p, bits, w.flag);
    k_scan<<<1, 1024, 0, s>>>(w.flag, w.id, w.parent, w.nodes, w.total);
    const long long next_bound = std::min<long long>(shots, 2LL * node_bound);
    k_project<T><<<(unsigned)next_bound, 128, 0, s>>>(Wm, w.p, w.parent, w.nodes, cr, (C*)w.v_next);
    k_advance<<<gs, 256, 0, s>>>(shots, n, q, bits, w.id, w.node_of);
    return cudaGetLastError();
}

template cudaError_t launch_sample_site<float>(const void*, int, int, const void*, int, int, int64_t, int,
                                               const double*, uint8_t*, SampleWork&, cudaStream_t);
template cudaError_t launch_sample_site<double>(const void*, int, int, const void*, int, int, int64_t, int,
                                                const double*, uint8_t*, SampleWork&, cudaStream_t);

}  // namespace tnsim
