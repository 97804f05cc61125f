// Batched one-sided (Hestenes) Jacobi SVD of theta for every gate of a launch.
//
// The paper decomposes theta with a Jacobi SVD (cusolverDnZgesvdj, Sec. IV.A);
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
// blocks once in round-robin ("circle") order: P - 1 rounds of P/2 disjoint block
// pairs.  A visit stages both blocks in shared memory, rotates the BC x BC cross
// pairs in BC rounds of BC disjoint pairs (one warp per pair, lanes over rows,
// warp-shuffle reductions; each warp keeps its block-I column in registers, and the
// column norms are tracked rather than recomputed per pair) and, in
// the first round of a sweep, the pairs inside each block as well, then writes the
// blocks back.  Each sweep therefore rotates every column pair exactly once.  A sweep
// that rotates nothing ends the gate's iteration; reaching max_sweeps sets ENOCONV.
//
// The launch is persistent: one CTA per SM (as occupancy allows) claims visits of
// any gate from a device-side queue, so gates of different sizes and all rounds of
// a layer share the machine without waves.  The visits of a round are independent;
// a gate's next round opens when the last visit of the current one is reported.  An
// idle CTA polls with a sleep; if nothing progresses for spin_limit polls (default
// 2^22, settable per state) it sets an error flag and leaves; every other CTA leaves
// at its next claim, abandoning the claim, and the unfinished gates report status 5
// (the host reports ETIMEOUT).  No other wait exists, and no CTA leaves with a copy
// in flight.
#include <float.h>

#include "jacobi_sched.cuh"
#include "tnsim_internal.h"

namespace tnsim {

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

// Rows owned by a lane in the register-resident layout: element k of a lane is row
// 64 (k / 2) + 2 lane + (k % 2), so each lane moves two consecutive rows with one
// 16-byte shared-memory access.
__device__ __forceinline__ int reg_row(int lane, int k) { return 64 * (k >> 1) + 2 * lane + (k & 1); }

// Rotation of a column pair whose first column lives in registers (layout above) and
// whose second column lives in shared memory: the second column is read once, kept in
// registers for the update and written back once (FULL: m == 32 * RPL, so no row needs
// a bounds test).  The two column norms are tracked instead of recomputed: a (the
// register column's, in a register) and *bj (the shared column's, in shared memory).
// Only g = x_i^H x_j is formed; after a rotation the norms are a - t|g| and b + t|g|
// (the eigenvalues of the pair's 2 x 2 Gram matrix).  The caller recomputes both
// exactly when a visit starts, so the tracked values drift over at most BC rotations.
template <typename T, typename C, int RPL, bool FULL>
__device__ __forceinline__ int rotate_reg_tracked(C (&xi)[RPL], C* __restrict__ xjs, int m, int lane, T tol2, T zthr,
                                                  T& a, T* bj) {
    C xj[RPL];
    T gr = 0, gi = 0;
#pragma unroll
    for (int k = 0; k < RPL; k += 2) {
        const int r = reg_row(lane, k);
        if (FULL || r < m) {
            if constexpr (sizeof(C) == 8) {
                const float4 v = *reinterpret_cast<const float4*>(xjs + r);
                xj[k].x = v.x; xj[k].y = v.y; xj[k + 1].x = v.z; xj[k + 1].y = v.w;
            } else {
                xj[k] = xjs[r];
                xj[k + 1] = xjs[r + 1];
            }
        } else {
            xj[k].x = 0; xj[k].y = 0; xj[k + 1].x = 0; xj[k + 1].y = 0;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const C u = xi[k + e], v = xj[k + e];
            gr = fma(u.x, v.x, fma(u.y, v.y, gr));
            gi = fma(u.x, v.y, fma(-u.y, v.x, gi));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
        gi += __shfl_xor_sync(0xffffffffu, gi, o);
    }
    const T b = *bj;
    T cm1, sr, si, tg;
    if (!rot_params_fast(a, b, gr, gi, tol2, zthr, cm1, sr, si, tg)) return 0;
    a -= tg;
    __syncwarp();
    if (lane == 0) *bj = b + tg;
#pragma unroll
    for (int k = 0; k < RPL; k += 2) {
        const int r = reg_row(lane, k);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const C u = xi[k + e], v = xj[k + e];
            C nu, nv;
            nu.x = u.x + fma(-si, v.y, fma(-sr, v.x, cm1 * u.x));
            nu.y = u.y + fma(si, v.x, fma(-sr, v.y, cm1 * u.y));
            nv.x = v.x + fma(-si, u.y, fma(sr, u.x, cm1 * v.x));
            nv.y = v.y + fma(si, u.x, fma(sr, u.y, cm1 * v.y));
            xi[k + e] = nu;
            xj[k + e] = nv;
        }
        if (FULL || r < m) {
            if constexpr (sizeof(C) == 8) {
                *reinterpret_cast<float4*>(xjs + r) = make_float4(xj[k].x, xj[k].y, xj[k + 1].x, xj[k + 1].y);
            } else {
                xjs[r] = xj[k];
                xjs[r + 1] = xj[k + 1];
            }
        }
    }
    return 1;
}

// squared norm of a register column (reg_row layout), summed over the warp
template <typename T, typename C, int RPL>
__device__ __forceinline__ T reg_norm2(const C (&x)[RPL]) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < RPL; ++k) a = fma(x[k].x, x[k].x, fma(x[k].y, x[k].y, a));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// shared-memory block back to W (L2 stores) by the threads from first_thread on
template <typename C>
__device__ __forceinline__ void copy_block_out_from(C* dst, const C* src, int count, int first_thread) {
    const int units = (int)((size_t)count * sizeof(C) / 16);
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    const int nt = (int)blockDim.x - first_thread;
    for (int i = (int)threadIdx.x - first_thread; i < units; i += nt) __stcg(d + i, s[i]);
}

// Persistent kernel: every CTA repeatedly claims one visit (gate g, global round
// number, block pair v) from the gates' claim words, processes it, and reports it.
// The last visit of a round advances that gate to its next round (and, at the end
// of a sweep, decides convergence).  Gates are scanned in descriptor order, which
// the host sorts by decreasing size.  A CTA never waits while holding a claim, so
// a CTA with nothing to claim only waits for work that running CTAs are doing.
template <typename T, int BC, int RPL, int MINB>
__global__ void __launch_bounds__(BC * 32, MINB)
k_jacobi(const GateDesc* __restrict__ gd, int n_gates, int n_lead, double tol_in, int max_sweeps,
         JacobiCtl* __restrict__ ctl, unsigned spin_limit) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* X = reinterpret_cast<C*>(smem_raw);       // [2*BC][m], column-major
    __shared__ int s_g, s_rnd, s_v, s_exit, s_rot, s_vis;
    __shared__ T s_bn[BC];                       // tracked squared norms of block J's columns
    __shared__ short s_V[kScanTable];            // visits per round of each gate

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned spins = 0, last_progress = 0;
    // where this CTA starts scanning: spread over the n_lead leading gates (those as large
    // as the first; the descriptors come sorted by decreasing size), so the CTAs share out
    // the largest gates instead of crowding the first ones; afterwards the gate it last
    // claimed, and from there on in descriptor order
    int scan0 = (int)(((long long)blockIdx.x * n_lead) / gridDim.x);
    for (int g = threadIdx.x; g < n_gates && g < kScanTable; g += blockDim.x)
        s_V[g] = (short)tour_of<BC>(gd[g]).V;
    __syncthreads();

    int have_next = 0, nxt_g = -1, nxt_rnd = 0, nxt_v = 0;   // warp 0: a claim made during the last visit
    int nxt_err = 0;                                          // the error flag read during the last visit
    for (;;) {
        if (warp == 0) {
            int found = 0, fg = -1, frnd = 0, fv = 0, err = 0;
            if (have_next) {
                found = 1;
                fg = nxt_g;
                frnd = nxt_rnd;
                fv = nxt_v;
                err = nxt_err;
                have_next = 0;
            } else {
                if (lane == 0) err = *((volatile int*)&ctl->error);
                claim_scan<BC>(gd, n_gates, s_V, scan0, lane, found, fg, frnd, fv);
            }
            if (found) scan0 = fg;
            if (lane == 0) {
                s_exit = 0;
                s_g = found ? fg : -1;
                s_rnd = frnd;
                s_v = fv;
                // after a timeout every CTA leaves, a claim in hand included: the gates
                // left unfinished report status 5
                if (err || (!found && (*((volatile int*)&ctl->n_finished) >= n_gates ||
                                       *((volatile int*)&ctl->error))))
                    s_exit = 1;
                s_rot = 0;
                s_vis = 0;
            }
        }
        __syncthreads();
        if (s_exit) break;
        if (s_g < 0) {
            if (threadIdx.x == 0) {
                const unsigned p = *((volatile unsigned*)&ctl->progress);
                if (p != last_progress) {
                    last_progress = p;
                    spins = 0;
                } else if (++spins > spin_limit) {
                    atomicExch(&ctl->error, 1);
                }
                __nanosleep(256);
            }
            __syncthreads();
            continue;
        }
        __threadfence();   // order the claim before reading the blocks of the previous round

        const int g = s_g, rnd = s_rnd, v = s_v;
        const GateDesc& d = gd[g];
        GateOut* out = d.out;
        const Tour tg = tour_of<BC>(d);
        const int m = tg.m, n = tg.n, nb = tg.nb, P = tg.P, R = tg.R;
        const int sweep = rnd / R, round = rnd - sweep * R;
        C* Wm = (C*)d.W;
        // default tolerance: FP64, sqrt(m) * eps (LAPACK's one-sided Jacobi uses the same
        // scale), floored at 4 eps for tiny m; FP32, 2 eps.  Near convergence the columns
        // are almost orthogonal, so the FP32 partial sums of g stay small and its rounding
        // error is a fraction of eps sqrt(a b): the tighter test is resolvable, and it
        // matters because a pair left non-orthogonal at tol tilts the kept subspace by
        // about tol / (relative gap at the cut).  A column below eps*sqrt(max(m,n))*|theta|_F
        // is zero.
        const double tol = tol_in > 0.0 ? tol_in
                                        : (sizeof(T) == 4 ? 2.0 * Eps<T>::v : fmax(sqrt((double)m), 4.0) * Eps<T>::v);
        const T tol2 = (T)(tol * tol);
        const T zthr = (T)(Eps<T>::v * Eps<T>::v * (double)max(m, n) * out->frob2);

        int I, J;
        if (nb == 1) {
            I = 0;
            J = -1;
        } else {
            rr_pair(P, round, v, I, J);
            if (I >= nb) { I = J; J = -1; }
            else if (J >= nb) J = -1;
            if (J >= 0 && J < I) { const int t = I; I = J; J = t; }
        }
        const bool intra = (round == 0);
        int my_rot = 0, my_vis = 0;
        if (J >= 0 || intra) {
            const int colI = I * BC, nI = min(BC, n - colI);
            const int colJ = J >= 0 ? J * BC : 0, nJ = J >= 0 ? min(BC, n - colJ) : 0;
            copy_blocks_in(X, Wm + (size_t)colI * m, nI * m, X + (size_t)BC * m, Wm + (size_t)colJ * m,
                           J >= 0 ? nJ * m : 0);
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
                        my_rot += rotate_pair<T>(X + (size_t)(base + a) * m, X + (size_t)(base + b) * m,
                                                 m, lane, tol2, zthr);
                    }
                    __syncthreads();
                }
            }
            if (J >= 0) {
                // cross pairs: warp w keeps column I_w in registers and meets every
                // column of J once, J_{(w + sft) mod BC} in round sft
                C xi[RPL];
                const C* ci = X + (size_t)warp * m;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int r = reg_row(lane, k);
                    if (warp < nI && r < m) {
                        xi[k] = ci[r];
                    } else {
                        xi[k].x = 0;
                        xi[k].y = 0;
                    }
                }
                const bool full = (m == 32 * RPL);
                // exact norms at the start of the cross pairs: a of the register column,
                // s_bn[w] of block J's column w
                T a_i = reg_norm2<T, C, RPL>(xi);
                if (warp < nJ) {
                    const C* cj = X + (size_t)(BC + warp) * m;
                    T bn = 0;
                    for (int r = lane; r < m; r += 32) bn = fma(cj[r].x, cj[r].x, fma(cj[r].y, cj[r].y, bn));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) bn += __shfl_xor_sync(0xffffffffu, bn, o);
                    if (lane == 0) s_bn[warp] = bn;
                }
                __syncthreads();
                for (int sft = 0; sft < BC; ++sft) {
                    const int b = (warp + sft) % BC;
                    if (warp < nI && b < nJ) {
                        my_vis += (lane == 0);
                        C* xjs = X + (size_t)(BC + b) * m;
                        my_rot += full ? rotate_reg_tracked<T, C, RPL, true>(xi, xjs, m, lane, tol2, zthr, a_i, &s_bn[b])
                                       : rotate_reg_tracked<T, C, RPL, false>(xi, xjs, m, lane, tol2, zthr, a_i, &s_bn[b]);
                    }
                    __syncthreads();
                }
                C* co = X + (size_t)warp * m;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int r = reg_row(lane, k);
                    if (warp < nI && r < m) co[r] = xi[k];
                }
                __syncthreads();
            }
            if (warp > 0) {
                copy_block_out_from(Wm + (size_t)colI * m, X, nI * m, 32);
                if (J >= 0) copy_block_out_from(Wm + (size_t)colJ * m, X + (size_t)BC * m, nJ * m, 32);
            }
        }
        // warp 0 claims the next visit while the other warps write the blocks back (a CTA
        // never waits while holding a claim, so claiming before this visit's report is safe)
        if (warp == 0) {
            int found, fg, frnd, fv;
            if (lane == 0) nxt_err = *((volatile int*)&ctl->error);
            claim_scan<BC>(gd, n_gates, s_V, scan0, lane, found, fg, frnd, fv);
            have_next = found;
            nxt_g = fg;
            nxt_rnd = frnd;
            nxt_v = fv;
        }
        if (lane == 0 && my_rot) atomicAdd(&s_rot, my_rot);
        if (lane == 0 && my_vis) atomicAdd(&s_vis, my_vis);
        __threadfence();   // every thread's block stores before the report
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_rot) {
                atomicAdd(&out->rot_sweep, s_rot);
                atomicAdd(&out->rotations, (unsigned long long)s_rot);
            }
            if (s_vis) atomicAdd(&out->visits, (unsigned long long)s_vis);
            __threadfence();
            const int dn = atomicAdd(&out->done, 1) + 1;
            if (dn == tg.V) {
                // last visit of this round: advance the gate
                out->done = 0;
                bool fin = false;
                if (round == R - 1) {
                    const int rs = atomicExch(&out->rot_sweep, 0);
                    if (rs == 0 || sweep + 1 >= max_sweeps) {
                        fin = true;
                        out->sweeps = sweep + 1;
                        // keep a timeout the contraction reported (5) before this launch
                        if (rs != 0 && out->status < 4) out->status = 4;
                    }
                }
                __threadfence();
                if (fin) {
                    atomicExch(&out->finished, 1);
                    atomicAdd(&ctl->n_finished, 1);
                } else {
                    atomicExch(&out->claim, (unsigned long long)(rnd + 1) << 32);
                }
                atomicAdd(&ctl->progress, 1u);
            }
        }
        __syncthreads();
    }
}

template <typename T, int BC, int RPL, int MINB>
static cudaError_t launch_bc(const GateDesc* d, int n_gates, int n_lead, int m_max, int n_max, double tol,
                             int max_sweeps, JacobiCtl* ctl, cudaStream_t s, unsigned spin_limit) {
    using C = typename CT<T>::type;
    const size_t smem = (size_t)2 * BC * m_max * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<T, BC, RPL, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi<T, BC, RPL, MINB>, BC * 32, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // no more CTAs than visits that can run at once
    const int nb = (n_max + BC - 1) / BC;
    const long long visits = (long long)n_gates * ((nb == 1) ? 1 : (nb + (nb & 1)) / 2);
    long long grid = (long long)sms * per_sm;
    if (grid > visits) grid = visits;
    if (grid < 1) grid = 1;
    const int lead = (n_lead < 1 || n_lead > n_gates) ? n_gates : n_lead;
    k_jacobi<T, BC, RPL, MINB><<<(unsigned)grid, BC * 32, smem, s>>>(d, n_gates, lead, tol,
                                                                      max_sweeps < 1 ? 1 : max_sweeps, ctl,
                                                                      spin_limit ? spin_limit : kSpinLimit);
    return cudaGetLastError();
}

// Block width BC and rows per lane RPL (= ceil(m_max / 32)) per precision: the two
// staged blocks take 2 BC m_max elements of shared memory (at most 128 KB).  Two
// configurations per shape: cfg 0 -- wide blocks, one CTA per SM (fewer rounds per
// sweep); cfg 1 -- half-width blocks, two CTAs per SM (independent barriers, twice
// the rounds).  Bit 1 of a state's configuration (QR preconditioning, k_qr.cu) does not
// change this launch.  tnsim_autotune times every configuration on a real layer.
template <typename T>
cudaError_t launch_jacobi(const GateDesc* d, int n_gates, int m_max, int n_max, double tol,
                          int max_sweeps, JacobiCtl* ctl, cudaStream_t s, int cfg, int n_lead,
                          unsigned spin_limit) {
    if (n_gates <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if ((cfg & 4) && m_max <= jacobi_tc_max_rows())
            return launch_jacobi_tc(d, n_gates, n_lead, n_max, tol, max_sweeps, ctl, s, spin_limit);
    }
    const bool narrow = (cfg & 1) != 0;
#define TNSIM_JAC(BC, RPL, MINB) launch_bc<T, BC, RPL, MINB>(d, n_gates, n_lead, m_max, n_max, tol, max_sweeps, ctl, s, spin_limit)
    if (m_max <= 64) return narrow ? TNSIM_JAC(8, 2, 2) : TNSIM_JAC(16, 2, 1);
    if (m_max <= 128) return narrow ? TNSIM_JAC(8, 4, 2) : TNSIM_JAC(16, 4, 1);
    if (m_max <= 256) return narrow ? TNSIM_JAC(8, 8, 2) : TNSIM_JAC(16, 8, 1);
    if constexpr (sizeof(T) == 4) {
        if (m_max <= 512) return narrow ? TNSIM_JAC(8, 16, 2) : TNSIM_JAC(16, 16, 1);
        return TNSIM_JAC(8, 32, 1);
    } else {
        if (m_max <= 512) return narrow ? TNSIM_JAC(4, 16, 2) : TNSIM_JAC(8, 16, 1);
        return TNSIM_JAC(4, 32, 1);
    }
#undef TNSIM_JAC
}

template cudaError_t launch_jacobi<float>(const GateDesc*, int, int, int, double, int, JacobiCtl*, cudaStream_t, int,
                                          int, unsigned);
template cudaError_t launch_jacobi<double>(const GateDesc*, int, int, int, double, int, JacobiCtl*, cudaStream_t, int,
                                           int, unsigned);

}  // namespace tnsim
