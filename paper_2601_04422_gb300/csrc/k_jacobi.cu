// Batched one-sided (Hestenes) Jacobi SVD of theta, one thread-block cluster per gate.
//
// The paper decomposes theta with a Jacobi SVD (cusolverDnZgesvdj, Sec. III.B);
// here the one-sided variant orthogonalises the n = 2chi_R columns of the
// m x n column-major working matrix W in place: W <- theta . V with V unitary,
// so at convergence the columns of W are u_j s_j.  V itself is never formed --
// the right site is recovered as U^H theta (see k_gemm.cu).
//
// Rotation of a column pair (i, j) (Hestenes 1958; Demmel & Veselic 1992, with
// the complex phase split off): a = |w_i|^2, b = |w_j|^2, g = w_i^H w_j = |g| e^{i phi}.
// If |g| > tol sqrt(a b):  zeta = (b - a) / (2|g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1+t^2), s = c t, and
//     w_i <- c w_i - s e^{-i phi} w_j,     w_j <- s e^{i phi} w_i + c w_j,
// which makes the pair orthogonal.  Columns whose norm is below
// eps*sqrt(max(m,n))*|theta|_F are numerically zero and are not rotated.
//
// Schedule.  The columns are cut into blocks of BC.  A sweep visits every pair of
// blocks once in round-robin ("circle") order; the P/2 block pairs of a round are
// spread over the CTAs of the gate's cluster, and a cluster barrier separates
// rounds (a block is touched by one CTA per round).  A visit stages both blocks in
// shared memory, rotates the BC x BC cross pairs in BC rounds of BC disjoint pairs
// (one warp per pair, lanes over rows, warp-shuffle reductions) and, in the first
// round of a sweep, the pairs inside each block as well, then writes the blocks
// back.  Each sweep therefore rotates every column pair exactly once.  A sweep that
// rotates nothing ends the iteration; reaching max_sweeps sets status ENOCONV.
// Every loop is bounded; the kernel never spins on memory.
#include <cooperative_groups.h>
#include <float.h>

#include "tnsim_internal.h"

namespace cg = cooperative_groups;

namespace tnsim {

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

// pair v of round r in the circle method for P players (P even)
__device__ __forceinline__ void rr_pair(int P, int r, int v, int& a, int& b) {
    if (v == 0) {
        a = P - 1;
        b = r;
    } else {
        a = (r + v) % (P - 1);
        b = (r - v + (P - 1)) % (P - 1);
    }
}

template <typename T, typename C>
__device__ __forceinline__ int rotate_pair(C* __restrict__ xi, C* __restrict__ xj, int m, int lane,
                                           T tol2, T zthr) {
    T a = 0, b = 0, gr = 0, gi = 0;
    for (int r = lane; r < m; r += 32) {
        const C u = xi[r], v = xj[r];
        a = fma(u.x, u.x, fma(u.y, u.y, a));
        b = fma(v.x, v.x, fma(v.y, v.y, b));
        gr = fma(u.x, v.x, fma(u.y, v.y, gr));
        gi = fma(u.x, v.y, fma(-u.y, v.x, gi));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
        gi += __shfl_xor_sync(0xffffffffu, gi, o);
    }
    const T g2 = gr * gr + gi * gi;
    if (!(a > zthr && b > zthr && g2 / b > tol2 * a)) return 0;
    const T gabs = sqrt(g2);
    const T zeta = (b - a) / (2 * gabs);
    const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
    // c = 1/rr, s = t/rr with rr = sqrt(1 + t^2), and c - 1 = -t^2 / (rr (1 + rr)) formed
    // directly.  Each new element is x + d, where the small correction d = (c-1) x + ...
    // is summed first and then added to x with a single rounding.  Near convergence
    // |(c-1) x| is below half an ulp of x: added to an already rounded x + ... it would
    // always round away, leaving c = 1 and growing the pair's norm by a factor 1 + t^2
    // per rotation (a systematic drift of the singular values in FP32).
    const T rr = sqrt(T(1) + t * t);
    const T cm1 = -(t * t) / (rr * (T(1) + rr));
    const T s = t / rr;
    const T er = gr / gabs, ei = gi / gabs;
    const T sr = s * er, si = s * ei;     // s e^{i phi}
    for (int r = lane; r < m; r += 32) {
        const C u = xi[r], v = xj[r];
        C nu, nv;
        // nu = c u - conj(s e) v = u + [(c-1) u - conj(s e) v]
        nu.x = u.x + fma(-si, v.y, fma(-sr, v.x, cm1 * u.x));
        nu.y = u.y + fma(si, v.x, fma(-sr, v.y, cm1 * u.y));
        // nv = (s e) u + c v = v + [(c-1) v + (s e) u]
        nv.x = v.x + fma(-si, u.y, fma(sr, u.x, cm1 * v.x));
        nv.y = v.y + fma(si, u.x, fma(sr, u.y, cm1 * v.y));
        xi[r] = nu;
        xj[r] = nv;
    }
    return 1;
}

template <typename C>
__device__ __forceinline__ void copy_block_in(C* dst, const C* src, int count) {
    const int units = (int)((size_t)count * sizeof(C) / 16);
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i = threadIdx.x; i < units; i += blockDim.x) d[i] = __ldcg(s + i);
}
template <typename C>
__device__ __forceinline__ void copy_block_out(C* dst, const C* src, int count) {
    const int units = (int)((size_t)count * sizeof(C) / 16);
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i = threadIdx.x; i < units; i += blockDim.x) __stcg(d + i, s[i]);
}

template <typename T, int BC>
__global__ void __launch_bounds__(BC * 32, 1)
k_jacobi(const GateDesc* __restrict__ gd, int CL, double tol_in, int max_sweeps) {
    using C = typename CT<T>::type;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int g = blockIdx.x / CL;
    const GateDesc& d = gd[g];
    const int chiL = d.chi[d.q], chiR = d.chi[d.q + 2];
    const int m = 2 * chiL, n = 2 * chiR;
    C* Wm = (C*)d.W;
    GateOut* out = d.out;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* X = reinterpret_cast<C*>(smem_raw);       // [2*BC][m], column-major
    __shared__ int s_rot;
    __shared__ unsigned long long s_vis;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = (n + BC - 1) / BC;
    const int P = nb + (nb & 1);
    // default tolerance sqrt(m) * eps (LAPACK's one-sided Jacobi uses the same scale),
    // floored at 4 eps for tiny m; a column below eps*sqrt(max(m,n))*|theta|_F is zero
    const double tol = tol_in > 0.0 ? tol_in : fmax(sqrt((double)m), 4.0) * Eps<T>::v;
    const T tol2 = (T)(tol * tol);
    const T zthr = (T)(Eps<T>::v * Eps<T>::v * (double)max(m, n) * out->frob2);

    if (crank == 0 && threadIdx.x == 0) {
        out->rot_ctr[0] = 0;
        out->rot_ctr[1] = 0;
        out->rot_ctr[2] = 0;
    }
    if (threadIdx.x == 0) s_vis = 0;
    __threadfence();
    cluster.sync();

    int sweep = 0;
    bool converged = false;
    unsigned long long total_rot = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        if (crank == 0 && threadIdx.x == 0) out->rot_ctr[(sweep + 1) % 3] = 0;
        __syncthreads();
        int my_rot = 0, my_vis = 0;
        const int rounds = (nb == 1) ? 1 : P - 1;
        for (int rnd = 0; rnd < rounds; ++rnd) {
            const int pairs = (nb == 1) ? 1 : P / 2;
            for (int v = crank; v < pairs; v += CL) {
                int I, J;
                if (nb == 1) { I = 0; J = -1; }
                else {
                    rr_pair(P, rnd, v, I, J);
                    if (I >= nb) { I = J; J = -1; }
                    else if (J >= nb) J = -1;
                    if (J >= 0 && J < I) { int t = I; I = J; J = t; }
                }
                const bool intra = (rnd == 0);
                if (J < 0 && !intra) continue;
                const int colI = I * BC, nI = min(BC, n - colI);
                const int colJ = J >= 0 ? J * BC : 0, nJ = J >= 0 ? min(BC, n - colJ) : 0;
                copy_block_in(X, Wm + (size_t)colI * m, nI * m);
                if (J >= 0) copy_block_in(X + (size_t)BC * m, Wm + (size_t)colJ * m, nJ * m);
                __syncthreads();
                if (intra) {
                    // pairs inside block I (warps 0..BC/2-1) and inside block J (the rest)
                    for (int t = 0; t < BC - 1; ++t) {
                        const int half = BC / 2;
                        const int w = warp < half ? warp : warp - half;
                        const int base = warp < half ? 0 : BC;
                        const int nblk = warp < half ? nI : nJ;
                        int a, b;
                        rr_pair(BC, t, w, a, b);
                        if (a < nblk && b < nblk) {
                            my_vis += (lane == 0);
                            my_rot += rotate_pair<T>(X + (size_t)(base + a) * m,
                                                     X + (size_t)(base + b) * m, m, lane, tol2, zthr);
                        }
                        __syncthreads();
                    }
                }
                if (J >= 0) {
                    for (int sft = 0; sft < BC; ++sft) {
                        const int a = warp, b = (warp + sft) % BC;
                        if (a < nI && b < nJ) {
                            my_vis += (lane == 0);
                            my_rot += rotate_pair<T>(X + (size_t)a * m, X + (size_t)(BC + b) * m, m,
                                                     lane, tol2, zthr);
                        }
                        __syncthreads();
                    }
                }
                copy_block_out(Wm + (size_t)colI * m, X, nI * m);
                if (J >= 0) copy_block_out(Wm + (size_t)colJ * m, X + (size_t)BC * m, nJ * m);
                __syncthreads();
            }
            __threadfence();
            cluster.sync();
        }
        if (lane == 0 && my_rot) atomicAdd(&s_rot, my_rot);
        if (lane == 0 && my_vis) atomicAdd(&s_vis, (unsigned long long)my_vis);
        __syncthreads();
        if (threadIdx.x == 0 && s_rot) atomicAdd(&out->rot_ctr[sweep % 3], s_rot);
        total_rot += (threadIdx.x == 0) ? (unsigned long long)s_rot : 0ull;
        __threadfence();
        cluster.sync();
        const int tot = *((volatile int*)&out->rot_ctr[sweep % 3]);
        if (tot == 0) { converged = true; ++sweep; break; }
    }
    if (threadIdx.x == 0) {
        if (total_rot) atomicAdd(&out->rotations, total_rot);
        if (s_vis) atomicAdd(&out->visits, s_vis);
        if (crank == 0) {
            out->sweeps = sweep;
            out->status = converged ? 0 : 4;
        }
    }
}

template <typename T, int BC>
static cudaError_t launch_bc(const GateDesc* d, int n_gates, int m_max, int n_max, double tol,
                             int max_sweeps, cudaStream_t s) {
    using C = typename CT<T>::type;
    const size_t smem = (size_t)2 * BC * m_max * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<T, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int nb = (n_max + BC - 1) / BC;
    const int pairs = (nb + (nb & 1)) / 2;
    int CL = 1;
    while (CL < 8 && CL < pairs) CL <<= 1;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    for (;;) {
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(n_gates * CL, 1, 1);
        cfg.blockDim = dim3(BC * 32, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int max_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&max_clusters, k_jacobi<T, BC>, &cfg);
        if (e == cudaSuccess && max_clusters > 0) break;
        (void)cudaGetLastError();
        if (CL == 1) return e == cudaSuccess ? cudaErrorLaunchOutOfResources : e;
        CL >>= 1;
    }
    return cudaLaunchKernelEx(&cfg, k_jacobi<T, BC>, d, CL, tol, max_sweeps);
}

template <typename T>
cudaError_t launch_jacobi(const GateDesc* d, int n_gates, int m_max, int n_max, double tol,
                          int max_sweeps, cudaStream_t s) {
    using C = typename CT<T>::type;
    if (n_gates <= 0) return cudaSuccess;
    const size_t budget = 200 * 1024;
    if ((size_t)2 * 16 * m_max * sizeof(C) <= budget)
        return launch_bc<T, 16>(d, n_gates, m_max, n_max, tol, max_sweeps, s);
    if ((size_t)2 * 8 * m_max * sizeof(C) <= budget)
        return launch_bc<T, 8>(d, n_gates, m_max, n_max, tol, max_sweeps, s);
    return launch_bc<T, 4>(d, n_gates, m_max, n_max, tol, max_sweeps, s);
}

template cudaError_t launch_jacobi<float>(const GateDesc*, int, int, int, double, int, cudaStream_t);
template cudaError_t launch_jacobi<double>(const GateDesc*, int, int, int, double, int, cudaStream_t);

}  // namespace tnsim
