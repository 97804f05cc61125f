// QR preconditioning of the Jacobi SVD (one-sided Jacobi on R^H, Drmac and Veselic,
// "New fast and accurate Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl. 29, 2008).
//
// For a square gated block theta = Q R (m = n), the one-sided Jacobi runs on the
// columns of R^H instead of theta's: it needs fewer sweeps (on saturated Haar
// brickwork gate blocks, 10.6 against 13.7 per gate at chi 256).  Q is never formed.  With W' = R^H V' the
// converged columns (W' = U'' S, U'' orthonormal), R = V' S U''^H, so
//   theta = (Q V') S U''^H:  the right singular vectors of theta are the columns of
//   U'' = W' S^-1, and
//   right site (the paper's S V^H) = rows (W'_j)^H  -- a gather (k_right_pre),
//   left site  U = theta V S^-1 = theta W' S^-2      -- one GEMM (k_left_pre).
//
// k_qr: blocked Householder QR, in place on W (a copy of theta), which becomes R^H
// (lower triangular, zeros above).  Panels of NB columns sit in shared memory; a panel
// is factorised column by column (reflectors H = I - tau v v^H with v_0 = 1 and real
// tau, Hermitian and unitary; H x = beta e_1 with beta = -e^{i arg x_0} |x|), then
// accumulated into the compact WY form H_0 ... H_{NB-1} = I - V T V^H (T upper
// triangular, built column by column from V^H V), and the trailing columns take
// A <- A - V T^H (V^H A): warp tasks of WC columns, V^H A reduced over the lanes by a
// reduce-scatter.  The rows of R a panel finishes are written conjugated straight into
// their R^H columns (the panel columns, dead once loaded).  Each gate runs on a cluster
// of G CTAs: every CTA factorises the panel redundantly (same data, same arithmetic,
// same result) and takes every G-th group of trailing tasks; two cluster barriers per
// panel order the writes into the panel columns after every copy of the panel, and the
// next panel's loads after every trailing write.
#include <algorithm>

#include "tnsim_internal.h"

namespace tnsim {

namespace {

template <typename C> __device__ __forceinline__ C cz() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> __device__ __forceinline__ void cmac(C& acc, const C& a, const C& b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename C> __device__ __forceinline__ void cmacc(C& acc, const C& a, const C& b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <typename C> __device__ __forceinline__ void cmsub(C& acc, const C& a, const C& b) {  // acc -= a b
    acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
// reduce-scatter of N values over the 32 lanes: afterwards v[t] (t < F) of lane L holds
// the lane sum of the value with index t + F L
template <int N, int F, typename C>
__device__ __forceinline__ void bfly(C* v, int lane) {
    if constexpr (N > F) {
        constexpr int H = N / 2, O = H / F;
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int t = 0; t < H; ++t) {
            const C lo = v[t], hi = v[t + H];
            const C send = up ? lo : hi;
            C keep = up ? hi : lo;
            keep.x += __shfl_xor_sync(0xffffffffu, send.x, O);
            keep.y += __shfl_xor_sync(0xffffffffu, send.y, O);
            v[t] = keep;
        }
        bfly<H, F>(v, lane);
    }
}

constexpr int QT = 256;   // threads of a CTA
constexpr int QW = QT / 32;
constexpr int WC = 4;     // trailing columns of one warp task

// cluster registers: this CTA's rank, the cluster's CTA count, the cluster index (the gate)
__device__ __forceinline__ unsigned cl_rank() { unsigned r; asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r)); return r; }
__device__ __forceinline__ unsigned cl_size() { unsigned r; asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r)); return r; }
__device__ __forceinline__ unsigned cl_id() { unsigned r; asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r)); return r; }
// every thread of the cluster; orders the global and shared accesses before it (release)
// before those after it (acquire), at cluster scope
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// global load cached in L2 only: the data may come from another CTA of the cluster
template <typename C> __device__ __forceinline__ C ldcg(const C* p) {
    if constexpr (sizeof(C) == 8) { float2 v = __ldcg(reinterpret_cast<const float2*>(p)); return *reinterpret_cast<C*>(&v); }
    else { double2 v = __ldcg(reinterpret_cast<const double2*>(p)); return *reinterpret_cast<C*>(&v); }
}

template <typename T, int NB>
__global__ void __launch_bounds__(QT, 1) k_qr(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    constexpr int NV = NB * WC, F = NV / 32;
    static_assert(NV % 32 == 0, "reduce-scatter needs a multiple of 32 values");
    const GateDesc& d = gd[cl_id()];
    const int rank = (int)cl_rank(), G = (int)cl_size();
    const int q = d.q;
    const int m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    if (!qr_active(d, m, n)) return;     // uniform over the cluster
    C* A = (C*)d.W;
    extern __shared__ __align__(16) unsigned char qr_smem[];
    C* Vp = reinterpret_cast<C*>(qr_smem);        // [NB][L0]
    __shared__ C Tm[NB][NB + 1], Zm[NB][NB + 1];
    __shared__ C s_sc[NB], s_beta[NB];
    __shared__ T s_tau[NB], s_sig[NB + 1];
    __shared__ C Ys[QW][NV], Zs[QW][NV];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int p0 = 0; p0 < n; p0 += NB) {
        const int nbp = min(NB, n - p0), L0 = m - p0;
        // ---- panel into shared memory (its columns were last written by the previous panel's
        // trailing update, possibly in another CTA of the cluster)
        for (int c = warp; c < NB; c += QW) {
            C* dst = Vp + (size_t)c * L0;
            if (c < nbp) {
                const C* src = A + (size_t)(p0 + c) * m + p0;
                int r = lane;
                for (; r + 96 < L0; r += 128) {
                    const C x0 = ldcg(src + r), x1 = ldcg(src + r + 32), x2 = ldcg(src + r + 64), x3 = ldcg(src + r + 96);
                    dst[r] = x0; dst[r + 32] = x1; dst[r + 64] = x2; dst[r + 96] = x3;
                }
                for (; r < L0; r += 32) dst[r] = ldcg(src + r);
            } else {
                for (int r = lane; r < L0; r += 32) dst[r] = cz<C>();
            }
        }
        if (rank == 0) {
            for (int c = warp; c < nbp; c += QW)
                for (int r = lane; r < p0; r += 32) A[(size_t)(p0 + c) * m + r] = cz<C>();
        }
        // every CTA of the cluster holds its copy of the panel before any writes R^H into it
        cl_sync();
        if (warp == 0) {
            T s = 0;
            for (int r = 1 + lane; r < L0; r += 32) s += Vp[r].x * Vp[r].x + Vp[r].y * Vp[r].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) s_sig[0] = s;
        }
        __syncthreads();
        // ---- panel factorisation: reflector j, applied to the panel columns right of it
        for (int j = 0; j < nbp; ++j) {
            const C alpha = Vp[(size_t)j * L0 + j];
            const T sigma = s_sig[j];
            T tau = 0;
            C sc = cz<C>(), beta = alpha;
            if (sigma > (T)0) {
                const T an = sqrt(alpha.x * alpha.x + alpha.y * alpha.y);
                const T xn = sqrt(an * an + sigma);
                const T px = an > (T)0 ? alpha.x / an : (T)1, py = an > (T)0 ? alpha.y / an : (T)0;
                const T v0m = an + xn;
                beta.x = -px * xn;
                beta.y = -py * xn;
                sc.x = px / v0m;
                sc.y = -py / v0m;
                tau = (T)2 / ((T)1 + sigma / (v0m * v0m));
            }
            if (tid == 0) { s_tau[j] = tau; s_sc[j] = sc; s_beta[j] = beta; }
            const C* x = Vp + (size_t)j * L0;
            for (int c = j + 1 + warp; c < nbp; c += QW) {
                C* y = Vp + (size_t)c * L0;
                C dot = cz<C>();
                for (int r = j + 1 + lane; r < L0; r += 32) cmacc(dot, x[r], y[r]);
                dot = warp_sum(dot);
                const C yj = y[j];
                C w;   // tau (v^H y), v = (1, sc x_{j+1..})
                w.x = tau * (sc.x * dot.x + sc.y * dot.y + yj.x);
                w.y = tau * (sc.x * dot.y - sc.y * dot.x + yj.y);
                C sw;
                sw.x = sc.x * w.x - sc.y * w.y;
                sw.y = sc.x * w.y + sc.y * w.x;
                __syncwarp();
                if (lane == 0) { y[j].x = yj.x - w.x; y[j].y = yj.y - w.y; }
                T nrm = 0;
                for (int r = j + 1 + lane; r < L0; r += 32) {
                    C v = y[r];
                    cmsub(v, x[r], sw);
                    y[r] = v;
                    if (r > c) nrm += v.x * v.x + v.y * v.y;
                }
                if (c == j + 1) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
                    if (lane == 0) s_sig[c] = nrm;
                }
            }
            __syncthreads();
        }
        for (int j = nbp + tid; j < NB; j += QT) s_tau[j] = 0;
        // ---- R^H of the panel block out (one CTA); reflectors scaled; unit diagonal, zeros above
        for (int c = warp; c < NB; c += QW) {
            C* col = Vp + (size_t)c * L0;
            const C s = c < nbp ? s_sc[c] : cz<C>();
            for (int r = lane; r < L0; r += 32) {
                C v = col[r];
                if (r < c) {
                    if (c < nbp && rank == 0) {
                        A[(size_t)(p0 + r) * m + p0 + c] = cconj(v);    // (R^H)[p0+c][p0+r]
                        A[(size_t)(p0 + c) * m + p0 + r] = cz<C>();
                    }
                    v = cz<C>();
                } else if (r == c) {
                    if (c < nbp && rank == 0) A[(size_t)(p0 + c) * m + p0 + c] = cconj(s_beta[c]);
                    v.x = c < nbp ? (T)1 : (T)0;
                    v.y = 0;
                } else {
                    C t;
                    t.x = v.x * s.x - v.y * s.y;
                    t.y = v.x * s.y + v.y * s.x;
                    v = t;
                }
                col[r] = v;
            }
        }
        __syncthreads();
        // ---- T of the compact WY form (forward, columnwise): Zm = V^H V above the diagonal
        for (int pidx = warp; pidx < NB * NB; pidx += QW) {
            const int i = pidx / NB, j = pidx - i * NB;
            if (i >= j) continue;
            C z = cz<C>();
            for (int r = j + lane; r < L0; r += 32) cmacc(z, Vp[(size_t)i * L0 + r], Vp[(size_t)j * L0 + r]);
            z = warp_sum(z);
            if (lane == 0) Zm[i][j] = z;
        }
        __syncthreads();
        if (warp == 0 && lane < NB) {
            // lane i builds row i of T; the row stays in registers (fully unrolled loops),
            // so the recurrence's only shared-memory reads are the independent Zm entries
            const int i = lane;
            C trow[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                C t = cz<C>();
                if (i < j) {
                    C acc = cz<C>();
#pragma unroll
                    for (int l = 0; l < j; ++l)
                        if (l >= i) cmac(acc, trow[l], Zm[l][j]);
                    t.x = -s_tau[j] * acc.x;
                    t.y = -s_tau[j] * acc.y;
                } else if (i == j) {
                    t.x = s_tau[j];
                }
                trow[j] = t;
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) Tm[i][j] = trow[j];
        }
        __syncthreads();
        // ---- trailing update A <- (I - V T^H V^H) A, WC columns per warp task, the tasks
        // spread over the cluster; the panel's rows of the result are rows of R, written
        // conjugated into R^H
        const int c_lo = p0 + nbp, nt = n - c_lo;
        for (int task = rank * QW + warp; task * WC < nt; task += G * QW) {
            const int c0 = c_lo + task * WC;
            const int nv = min(WC, n - c0);
            C v[NV];
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = cz<C>();
            C* aw = A + (size_t)c0 * m + p0;
            C an[WC];
#pragma unroll
            for (int c = 0; c < WC; ++c) an[c] = (c < nv && lane < L0) ? ldcg(aw + (size_t)c * m + lane) : cz<C>();
            for (int r = lane; r < L0; r += 32) {
                C a[WC];
#pragma unroll
                for (int c = 0; c < WC; ++c) a[c] = an[c];
                if (r + 32 < L0) {
#pragma unroll
                    for (int c = 0; c < WC; ++c) an[c] = c < nv ? ldcg(aw + (size_t)c * m + r + 32) : cz<C>();
                }
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const C vi = Vp[(size_t)i * L0 + r];
#pragma unroll
                    for (int c = 0; c < WC; ++c) cmacc(v[i * WC + c], vi, a[c]);
                }
            }
            bfly<NV, F>(v, lane);
#pragma unroll
            for (int t = 0; t < F; ++t) Ys[warp][F * lane + t] = v[t];
            __syncwarp();
#pragma unroll
            for (int t = 0; t < F; ++t) {
                const int f = F * lane + t, i = f / WC, c = f - i * WC;
                C z = cz<C>();
                for (int l = 0; l <= i; ++l) cmacc(z, Tm[l][i], Ys[warp][l * WC + c]);
                Zs[warp][f] = z;
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = Zs[warp][t];
#pragma unroll
            for (int c = 0; c < WC; ++c) an[c] = (c < nv && lane < L0) ? ldcg(aw + (size_t)c * m + lane) : cz<C>();
            for (int r = lane; r < L0; r += 32) {
                C a[WC];
#pragma unroll
                for (int c = 0; c < WC; ++c) a[c] = an[c];
                if (r + 32 < L0) {
#pragma unroll
                    for (int c = 0; c < WC; ++c) an[c] = c < nv ? ldcg(aw + (size_t)c * m + r + 32) : cz<C>();
                }
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const C vi = Vp[(size_t)i * L0 + r];
#pragma unroll
                    for (int c = 0; c < WC; ++c) cmsub(a[c], vi, v[i * WC + c]);
                }
                if (r < nbp) {
#pragma unroll
                    for (int c = 0; c < WC; ++c)
                        if (c < nv) A[(size_t)(p0 + r) * m + c0 + c] = cconj(a[c]);
                } else {
#pragma unroll
                    for (int c = 0; c < WC; ++c)
                        if (c < nv) aw[(size_t)c * m + r] = a[c];
                }
            }
            __syncwarp();
        }
        cl_sync();
    }
}

// left site U_k = theta W'_k S^-2: (m x n, theta0 column-major) times the kept
// Jacobi columns (n x k, column perm[j] of W divided by s_j^2); 64 x 64 tiles
template <typename T>
__global__ void __launch_bounds__(256) k_left_pre(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q, m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    if (!qr_active(d, m, n)) return;
    const int k = d.out->k;
    const int r0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    if (r0 >= m || j0 >= k) return;
    __shared__ C As[16][64];
    __shared__ C Bs[16][65];
    __shared__ int pj[64];
    __shared__ T fj[64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < 64) {
        const int j = j0 + tid;
        pj[tid] = j < k ? d.perm[j] : -1;
        const double s2 = j < k ? d.s2[j] : 0.0;
        fj[tid] = s2 > 0.0 ? (T)(1.0 / s2) : (T)0;
    }
    __syncthreads();
    const C* T0 = (const C*)d.theta0;
    const C* W = (const C*)d.W;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cz<C>();
    for (int c0 = 0; c0 < n; c0 += 16) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t;
            const int cc = e / 64, rr = e % 64;                 // theta tile: 16 columns x 64 rows
            As[cc][rr] = (c0 + cc < n && r0 + rr < m) ? T0[(size_t)(c0 + cc) * m + r0 + rr] : cz<C>();
            const int jj = e / 16, kc = e % 16;                 // W' tile: 64 kept columns x 16 rows
            C w = cz<C>();
            if (pj[jj] >= 0 && c0 + kc < n) {
                w = W[(size_t)pj[jj] * n + c0 + kc];
                w.x *= fj[jj];
                w.y *= fj[jj];
            }
            Bs[kc][jj] = w;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
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
    C* U = (C*)d.siteA;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx + 16 * j;
            if (jj < k) U[(size_t)r * k + jj] = acc[i][j];
        }
    }
}

// right site (the paper's S V^H, renormalised): row j = scale * (column perm[j] of W)^H
template <typename T>
__global__ void k_right_pre(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.y];
    const int q = d.q, m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    if (!qr_active(d, m, n)) return;
    const int k = d.out->k;
    const T sc = (T)d.out->scale;
    const C* W = (const C*)d.W;
    C* R = (C*)d.siteB;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * n; i += gridDim.x * blockDim.x) {
        const int j = i / n, c = i - j * n;
        C w = W[(size_t)d.perm[j] * n + c];
        C o;
        o.x = sc * w.x;
        o.y = -sc * w.y;
        R[i] = o;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_qr(const GateDesc* d, int n_gates, int m_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    constexpr int NB = sizeof(T) == 4 ? 16 : 8;
    using C = typename CT<T>::type;
    // gates with m > kQrMaxRows are not preconditioned (qr_active) and need no panel
    const size_t smem = (size_t)NB * std::min(m_max, kQrMaxRows) * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_qr<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(QT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // the widest cluster (at most 4 CTAs) with which every gate's cluster is resident at once
    int G = 1;
    for (int g = 4; g >= 2; --g) {
        at[0].val.clusterDim.x = g;
        cfg.gridDim = dim3(n_gates * g);
        int fit = 0;
        if (cudaOccupancyMaxActiveClusters(&fit, k_qr<T, NB>, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();   // a refused query only narrows the cluster
            continue;
        }
        if (fit >= n_gates) {
            G = g;
            break;
        }
    }
    at[0].val.clusterDim.x = G;
    cfg.gridDim = dim3(n_gates * G);
    e = cudaLaunchKernelEx(&cfg, k_qr<T, NB>, d);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sites_pre(const GateDesc* d, int n_gates, int m_max, int k_max, int n_max, cudaStream_t s,
                             int tc) {
    if (n_gates <= 0) return cudaSuccess;
    cudaError_t e;
    if (sizeof(T) == 4 && tc) {
        e = launch_left_pre_tc(d, n_gates, m_max, k_max, s);   // tensor cores (k_sites_tc.cu)
    } else {
        dim3 g1((m_max + 63) / 64, (k_max + 63) / 64, n_gates);
        k_left_pre<T><<<g1, 256, 0, s>>>(d);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)std::max(1, std::min(64, (k_max * n_max + 255) / 256)), n_gates);
    k_right_pre<T><<<g2, 256, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t launch_qr<float>(const GateDesc*, int, int, cudaStream_t);
template cudaError_t launch_qr<double>(const GateDesc*, int, int, cudaStream_t);
template cudaError_t launch_sites_pre<float>(const GateDesc*, int, int, int, int, cudaStream_t, int);
template cudaError_t launch_sites_pre<double>(const GateDesc*, int, int, int, int, cudaStream_t, int);

}  // namespace tnsim
