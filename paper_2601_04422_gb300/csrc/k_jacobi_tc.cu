// Complex64 one-sided Jacobi SVD whose visits rotate the block pair's Gram matrix and
// apply the accumulated rotation to the columns with tcgen05 tensor-core products.
//
// The schedule is k_jacobi.cu's: columns in blocks of BC = 16, every block pair visited
// once per sweep in round-robin order, a visit rotating the 16 x 16 cross pairs in 16
// steps of 16 disjoint pairs (and, in round 0, the pairs inside each block), a
// persistent launch claiming visits from the per-gate claim words.  What a visit of the
// blocks I, J (X = [X_I X_J], m x 32 columns of W) computes is the same sequence of
// Jacobi rotations (Sec. IV.A; Hestenes), with the inner products taken from the Gram
// matrix instead of the columns:
//   1. G = X^H X on the tensor cores: with Y = [Re X | Im X] (m x 64 real), the product
//      Y^T Y in 3xTF32 (hi.hi + hi.lo + lo.hi, FP32 accumulation in TMEM), each 128-row
//      operand tile holding 32 rows of each half of Y (the diagonal blocks of its
//      product are the two halves' contributions); Re G = P11 + P22, Im G = P12 - P21.
//   2. The visit's rotations on G: a pair (i, j) takes a = G_ii, b = G_jj, g = G_ij and
//      the rotation parameters of k_jacobi (every warp computes all 16 of a step and
//      shares them by shuffles); a step's rotations J (16 disjoint pairs) give
//      G <- J^H G J and D <- D J + (J - I), D = V - I the accumulated rotation minus the
//      identity.  Every new entry is its old value plus a correction summed first (the
//      single-rounding update of k_jacobi); the rotated pair's norms become a - t|g| and
//      b + t|g| and its coupling 0, as for the tracked norms there.
//   3. X <- X + X D on the tensor cores: [Re X | Im X] . [[Re D, Im D], [-Im D, Re D]]
//      in 3xTF32, chunks of 128 rows, the correction added to X in the epilogue (so a
//      column that barely moves keeps its bits).  A visit that rotates nothing writes
//      nothing back.
// Both blocks are staged in shared memory once per visit (asynchronous 16-byte copies),
// so m <= 512; the rotation steps touch only the 32 x 32 matrices.
//
// Operand tiles are written by the threads into 128-byte-swizzled K-major layout (the
// layout a SWIZZLE_128B TMA copy produces), made visible to the tensor cores with a
// proxy fence, and consumed by MMAs one thread issues; completion is signalled by
// tcgen05.commit on an mbarrier whose wait is bounded (GateDesc::wait_polls, default
// 2^26 polls).  A wait that runs out waits once more (bounded) for the MMAs in flight,
// sets the launch's error flag and the gate's status 5, and the CTA leaves after
// releasing its TMEM; every other CTA leaves at its next claim.
#include <float.h>

#include "jacobi_sched.cuh"
#include "tc_common.cuh"
#include "tnsim_internal.h"

namespace tnsim {

namespace {

constexpr int GB = 16;                 // columns per block
constexpr int GC = 2 * GB;             // complex columns of a visit
constexpr int GT = 512;                // threads of a CTA
constexpr int GS = GC + 1;             // row stride of the 32 x 32 matrices in shared memory
constexpr int GM = 512;                // largest m (rows) the staged blocks hold
constexpr unsigned kGramSpin = 1u << 26;

// dynamic shared memory (1024-byte aligned base)
constexpr uint32_t TILE128 = 128 * 128;                 // 128 rows x 128 bytes
constexpr uint32_t TILE64 = 64 * 128;                   // 64 rows x 128 bytes
constexpr uint32_t OFF_X = 0;                           // staged blocks: 32 columns x m complex
constexpr uint32_t OFF_T = GC * GM * 8;                 // 64 KB of tiles, 1024-aligned
// Gram phase: K-tile buffer b (hi, lo) at OFF_T + b * 2 TILE128; after it, P = Y^T Y
// (64 x 65 floats) at OFF_T.  Update phase: A tiles (hi, lo) of one K tile at OFF_T, the
// B tiles (K tile kt, hi / lo) at OFF_B + (2 kt + hl) TILE64.
constexpr uint32_t OFF_B = OFF_T + 2 * TILE128;
constexpr uint32_t OFF_G = OFF_T + 4 * TILE128;         // G: two buffers of 32 x 33 float2
constexpr uint32_t OFF_D = OFF_G + 2 * GC * GS * 8;     // D: 32 x 33 float2 (updated in place)
constexpr uint32_t SMEM_USED = OFF_D + GC * GS * 8;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;       // slack for aligning the base

// Pair w (0..15) of a step, q1 < q2.  Cross step sft: column w of block I and column
// (w + sft) mod 16 of block J.  Intra step t: the circle-method pairs of round t among
// the 16 columns of each block (rr_pair(16, t, .)), w < 8 in block I, w >= 8 in block J.
__device__ __forceinline__ void pair_of(int w, int step, bool intra, int& q1, int& q2) {
    if (!intra) {
        q1 = w;
        q2 = GB + (w + step) % GB;
        return;
    }
    const int base = w < GB / 2 ? 0 : GB;
    int a, b;
    rr_pair(GB, step, w & (GB / 2 - 1), a, b);
    q1 = base + min(a, b);
    q2 = base + max(a, b);
}

// Inverse of pair_of: the pair w of index x (0..31) in a step, and whether x is the
// pair's second (larger) index.
__device__ __forceinline__ void pair_index(int x, int step, bool intra, int& w, int& second) {
    if (!intra) {
        if (x < GB) {
            w = x;
            second = 0;
        } else {
            w = (x - GB - step + 2 * GB) % GB;
            second = 1;
        }
        return;
    }
    const int base = x < GB ? 0 : GB, y = x - base;
    int v, partner;
    if (y == GB - 1 || y == step) {
        v = 0;
        partner = y == step ? GB - 1 : step;
    } else {
        const int v1 = (y - step + (GB - 1)) % (GB - 1);
        v = v1 <= GB / 2 - 1 ? v1 : (step - y + (GB - 1)) % (GB - 1);
        partner = (2 * step - y + 2 * (GB - 1)) % (GB - 1);
    }
    w = (base ? GB / 2 : 0) + v;
    second = y > partner;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

__device__ __forceinline__ void st_split(unsigned char* hi_tile, unsigned char* lo_tile, uint32_t off, float v) {
    const float h = tf32_round(v);
    *reinterpret_cast<float*>(hi_tile + off) = h;
    *reinterpret_cast<float*>(lo_tile + off) = tf32_round(v - h);
}

// issue (one thread) the 3xTF32 products of one 32-wide K tile: D += Ahi Bhi + Ahi Blo + Alo Bhi
__device__ __forceinline__ void mma_ktile(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, uint32_t idesc, bool first) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t ah = smem_desc(a_hi + 32 * j), al = smem_desc(a_lo + 32 * j);
        const uint64_t bh = smem_desc(b_hi + 32 * j), bl = smem_desc(b_lo + 32 * j);
        mma_tf32(d_tmem, ah, bh, idesc, (first && j == 0) ? 0u : 1u);
        mma_tf32(d_tmem, ah, bl, idesc, 1u);
        mma_tf32(d_tmem, al, bh, idesc, 1u);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

}  // namespace

// Persistent kernel (protocol of k_jacobi: claim a visit, process it, report it; the
// last report of a round opens the gate's next round or ends its iteration).
__global__ void __launch_bounds__(GT, 1)
k_jacobi_tc(const GateDesc* __restrict__ gd, int n_gates, int n_lead, double tol_in, int max_sweeps,
            JacobiCtl* __restrict__ ctl, unsigned spin_limit) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float2* Xs = reinterpret_cast<float2*>(sm + OFF_X);    // column c of the visit at Xs + c m
    float* Ps = reinterpret_cast<float*>(sm + OFF_T);
    float2* Gb = reinterpret_cast<float2*>(sm + OFF_G);
    float2* Ds = reinterpret_cast<float2*>(sm + OFF_D);
    const uint32_t sbase = smem_u32(sm);
    __shared__ int s_g, s_rnd, s_v, s_exit, s_rot, s_vis, s_fail, s_ok;
    __shared__ short s_V[kScanTable];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned spins = 0, last_progress = 0;
    int scan0 = (int)(((long long)blockIdx.x * n_lead) / gridDim.x);
    for (int g = tid; g < n_gates && g < kScanTable; g += blockDim.x) s_V[g] = (short)tour_of<GB>(gd[g]).V;
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar[0]), 1);
        mbar_init(smem_u32(&s_bar[1]), 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t t_gram = s_tmem, t_upd = s_tmem + 128;   // 128 + 64 of the 256 columns held
    const uint32_t idesc = idesc_mn(2u, 0u, 128, 64), idesc_g = idesc_mn(2u, 0u, 128, 128);
    uint32_t ph[2] = {0u, 0u};         // (thread 0) parity of the next completion of each barrier
    bool pend[2] = {false, false};     // (thread 0) a commit on the barrier not yet waited for
    const uint32_t bar0 = smem_u32(&s_bar[0]), bar1 = smem_u32(&s_bar[1]);

    // (thread 0) bounded wait for the outstanding commit on barrier b; false on timeout
    auto wait_bar = [&](int b, unsigned lim) -> bool {
        if (!pend[b]) return true;
        const bool ok = mbar_wait(b ? bar1 : bar0, ph[b], lim);
        if (ok) {
            ph[b] ^= 1u;
            pend[b] = false;
        }
        return ok;
    };

    for (;;) {
        if (warp == 0) {
            int found = 0, fg = -1, frnd = 0, fv = 0, err = 0;
            if (lane == 0) err = *((volatile int*)&ctl->error) | s_fail;
            err = __shfl_sync(0xffffffffu, err, 0);
            if (!err) claim_scan<GB>(gd, n_gates, s_V, scan0, lane, found, fg, frnd, fv);
            if (found) scan0 = fg;
            if (lane == 0) {
                s_exit = 0;
                s_g = found ? fg : -1;
                s_rnd = frnd;
                s_v = fv;
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
            if (tid == 0) {
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
        __threadfence();

        const int g = s_g, rnd = s_rnd, v = s_v;
        const GateDesc& d = gd[g];
        GateOut* out = d.out;
        const Tour tgr = tour_of<GB>(d);
        const int m = tgr.m, n = tgr.n, nb = tgr.nb, P = tgr.P, R = tgr.R;
        const int sweep = rnd / R, round = rnd - sweep * R;
        float2* Wm = (float2*)d.W;
        const double tol = tol_in > 0.0 ? tol_in : 2.0 * Eps<float>::v;
        const float tol2 = (float)(tol * tol);
        const float zthr = (float)(Eps<float>::v * Eps<float>::v * (double)max(m, n) * out->frob2);
        const unsigned lim = d.wait_polls > 0 ? (unsigned)d.wait_polls : kGramSpin;

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
        bool fail = false;
        if (J >= 0 || intra) {
            const int colI = I * GB, nI = min(GB, n - colI);
            const int colJ = J >= 0 ? J * GB : 0, nJ = J >= 0 ? min(GB, n - colJ) : 0;
            auto valid = [&](int c) { return c < GB ? c < nI : c - GB < nJ; };
            copy_blocks_in(Xs, Wm + (size_t)colI * m, nI * m, Xs + (size_t)GB * m, Wm + (size_t)colJ * m,
                           J >= 0 ? nJ * m : 0);
            __syncthreads();
            // ---- 1. Gram products.  The rows are cut into two halves at h0 (a multiple of
            // 32); K tile kt holds rows kt*32.. of the first half in tile rows 0..63 and the
            // same rows of the second half in tile rows 64..127, and the 128 x 128 product
            // of the tile with itself has Y1^T Y1 and Y2^T Y2 on its diagonal blocks:
            // P = Y^T Y is their sum.  Every tile row carries data, and the MMA count is
            // half of what a 64-row tile padded to M = 128 would need.  Two tile buffers.
            const int nkt = (m + 63) / 64, h0 = 32 * nkt;
            for (int kt = 0; kt < nkt; ++kt) {
                const int b = kt & 1;
                if (tid == 0) s_ok = wait_bar(b, lim);   // the products of tile kt - 2 read this buffer
                __syncthreads();
                if (!s_ok) {
                    fail = true;
                    break;
                }
                unsigned char* hi = sm + OFF_T + b * 2 * TILE128;
                unsigned char* lo = hi + TILE128;
                {
                    const int c = tid >> 4, rr = (tid & 15) * 2;
                    const bool vc = valid(c);
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int row = half * h0 + kt * 32 + rr, t0 = half * 2 * GC;
                        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (vc && row < m) x = *reinterpret_cast<const float4*>(Xs + (size_t)c * m + row);
                        st_split(hi, lo, sw128_off(t0 + c, rr), x.x);
                        st_split(hi, lo, sw128_off(t0 + c, rr + 1), x.z);
                        st_split(hi, lo, sw128_off(t0 + GC + c, rr), x.y);
                        st_split(hi, lo, sw128_off(t0 + GC + c, rr + 1), x.w);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = sbase + OFF_T + b * 2 * TILE128, al = ah + TILE128;
                    mma_ktile(t_gram, ah, al, ah, al, idesc_g, kt == 0);
                    mma_commit(b ? bar1 : bar0);
                    pend[b] = true;
                }
            }
            if (!fail) {
                if (tid == 0) s_ok = wait_bar(0, lim) && wait_bar(1, lim);
                __syncthreads();
                fail = !s_ok;
            }
            if (!fail) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (warp < 4) {
                    // warps 0-1: rows 0..63, columns 0..63 (Y1^T Y1); warps 2-3: rows 64..127,
                    // columns 64..127 (Y2^T Y2), into two staging arrays
                    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
                    const int r = (warp & 1) * 32 + lane, c0 = (warp >> 1) * 64;
                    float* prow = Ps + (warp >> 1) * 64 * 65 + r * 65;
#pragma unroll
                    for (int cc = 0; cc < 64; cc += 16) {
                        float vv[16];
                        tmem_ld16(t_gram + lane_off + c0 + cc, vv);
#pragma unroll
                        for (int e = 0; e < 16; ++e) prow[cc + e] = vv[e];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                const float* P2 = Ps + 64 * 65;
                for (int e = tid; e < GC * GC; e += GT) {
                    const int i = e >> 5, j = e & 31;
                    const float gr = (Ps[i * 65 + j] + P2[i * 65 + j]) + (Ps[(GC + i) * 65 + GC + j] + P2[(GC + i) * 65 + GC + j]);
                    const float gi = (Ps[i * 65 + GC + j] + P2[i * 65 + GC + j]) - (Ps[(GC + i) * 65 + j] + P2[(GC + i) * 65 + j]);
                    Gb[i * GS + j] = make_float2(gr, gi);
                    Ds[i * GS + j] = make_float2(0.f, 0.f);
                }
                __syncthreads();
            }
            // ---- 2. the visit's rotations on G, accumulated in D = V - I
            int cur = 0;
            // One barrier per step: every warp computes all 16 pairs' rotation parameters
            // (lane w and lane w + 16: pair w; the same inputs and instructions in every
            // warp, so every warp reaches the same results and the same skip decision)
            // and hands them to its threads by shuffles.  A step that rotates nothing
            // changes nothing and needs no barrier.
            auto run_step = [&](int step, bool stin) {
                const float2* G = Gb + cur * GC * GS;
                int q1w, q2w;
                pair_of(lane & (GB - 1), step, stin, q1w, q2w);
                const bool exam = valid(q1w) && valid(q2w);
                float cmw = 0.f, srw = 0.f, siw = 0.f, tgw = 0.f;
                int rot = 0;
                if (exam) {
                    const float2 gq = G[q1w * GS + q2w];
                    rot = rot_params_fast(G[q1w * GS + q1w].x, G[q2w * GS + q2w].x, gq.x, gq.y, tol2, zthr, cmw, srw,
                                          siw, tgw);
                }
                const unsigned rb = __ballot_sync(0xffffffffu, rot), eb = __ballot_sync(0xffffffffu, exam);
                if (tid == 0) {
                    s_rot += __popc(rb & 0xffffu);
                    s_vis += __popc(eb & 0xffffu);
                }
                if (rb == 0u) return;   // G and D unchanged
                // thread: row p of G and D, the two columns q1 < q2 of pair w
                const int p = tid >> 4, w = tid & 15;
                int wp, psec;
                pair_index(p, step, stin, wp, psec);
                const float cq0 = __shfl_sync(0xffffffffu, cmw, w), sr = __shfl_sync(0xffffffffu, srw, w);
                const float si = __shfl_sync(0xffffffffu, siw, w), tq = __shfl_sync(0xffffffffu, tgw, w);
                const int rq = __shfl_sync(0xffffffffu, rot, w);
                const int q1 = __shfl_sync(0xffffffffu, q1w, w), q2 = __shfl_sync(0xffffffffu, q2w, w);
                const float cp0 = __shfl_sync(0xffffffffu, cmw, wp), srp = __shfl_sync(0xffffffffu, srw, wp);
                const float sip = __shfl_sync(0xffffffffu, siw, wp);
                const int rp = __shfl_sync(0xffffffffu, rot, wp);
                const int p1 = __shfl_sync(0xffffffffu, q1w, wp), p2 = __shfl_sync(0xffffffffu, q2w, wp);
                const int pp = psec ? p1 : p2;
                // J_{q2 q1} = -conj(s e), J_{q1 q2} = s e, J_qq = 1 + cm1 (zero factors if not rotated)
                const float cq = rq ? cq0 : 0.f;
                const float2 off1 = rq ? make_float2(-sr, si) : make_float2(0.f, 0.f);
                const float2 off2 = rq ? make_float2(sr, si) : make_float2(0.f, 0.f);
                const float cp = rp ? cp0 : 0.f;
                const float2 offp = rp ? (psec ? make_float2(srp, sip) : make_float2(-srp, sip))
                                       : make_float2(0.f, 0.f);   // J_{p' p}
                float2* Gn = Gb + (cur ^ 1) * GC * GS;
                const float2 a1 = G[p * GS + q1], a2 = G[p * GS + q2];
                const float2 b1 = G[pp * GS + q1], b2 = G[pp * GS + q2];
                // (G J)_{x q} = G_xq + H_xq
                const float2 ha1 = cadd(cscale(cq, a1), cmul(a2, off1)), ha2 = cadd(cscale(cq, a2), cmul(a1, off2));
                const float2 hb1 = cadd(cscale(cq, b1), cmul(b2, off1)), hb2 = cadd(cscale(cq, b2), cmul(b1, off2));
                // (J^H G J)_{pq} = G_pq + [H_pq + cm1_p (G J)_pq + conj(J_{p'p}) (G J)_{p'q}]
                float2 n1 = cadd(a1, cadd(cadd(ha1, cscale(cp, cadd(a1, ha1))), cmulc(offp, cadd(b1, hb1))));
                float2 n2 = cadd(a2, cadd(cadd(ha2, cscale(cp, cadd(a2, ha2))), cmulc(offp, cadd(b2, hb2))));
                if (rq && p == q1) {
                    n1 = make_float2(a1.x - tq, 0.f);
                    n2 = make_float2(0.f, 0.f);
                } else if (rq && p == q2) {
                    n1 = make_float2(0.f, 0.f);
                    n2 = make_float2(a2.x + tq, 0.f);
                }
                Gn[p * GS + q1] = n1;
                Gn[p * GS + q2] = n2;
                if (rq) {
                    // D <- D J + (J - I), in place (this thread alone owns D[p][q1], D[p][q2])
                    const float2 d1 = Ds[p * GS + q1], d2 = Ds[p * GS + q2];
                    float2 c1 = cadd(cscale(cq, d1), cmul(d2, off1));
                    float2 c2 = cadd(cscale(cq, d2), cmul(d1, off2));
                    if (p == q1) {
                        c1.x += cq;
                        c2 = cadd(c2, off2);
                    } else if (p == q2) {
                        c1 = cadd(c1, off1);
                        c2.x += cq;
                    }
                    Ds[p * GS + q1] = cadd(d1, c1);
                    Ds[p * GS + q2] = cadd(d2, c2);
                }
                __syncthreads();
                cur ^= 1;
            };
            if (!fail) {
                if (intra)
                    for (int t = 0; t < GB - 1; ++t) run_step(t, true);
                if (J >= 0)
                    for (int sft = 0; sft < GB; ++sft) run_step(sft, false);
                __syncthreads();   // s_rot complete; the last steps may have needed no barrier
            }
            // ---- 3. X <- X + X D on the tensor cores (only if anything rotated)
            if (!fail && s_rot > 0) {
                // B tiles: row n, K index k of R_D^T, R_D = [[Re D, Im D], [-Im D, Re D]] (K x N = 64 x 64)
                for (int e = tid; e < 64 * 64; e += GT) {
                    const int nn = e >> 6, k = e & 63;
                    const float2 dv = Ds[(k & 31) * GS + (nn & 31)];
                    const float val = k < GC ? (nn < GC ? dv.x : dv.y) : (nn < GC ? -dv.y : dv.x);
                    unsigned char* bh = sm + OFF_B + (k >> 5) * 2 * TILE64;
                    st_split(bh, bh + TILE64, sw128_off(nn, k & 31), val);
                }
                const int nrc = (m + 127) / 128;
                for (int rc = 0; rc < nrc && !fail; ++rc) {
                    const int r0 = rc * 128;
                    for (int kt = 0; kt < 2; ++kt) {
                        // A tile of K tile kt: row (matrix row - r0), K index c: Re X (kt 0) / Im X (kt 1)
                        {
                            unsigned char* ah = sm + OFF_T;
                            unsigned char* al = ah + TILE128;
                            // rows 16 h + (tid & 15): the 16 threads of a column store into
                            // rows of eight different swizzle phases (no 16-way bank conflict)
                            const int c = tid >> 4, rb = tid & 15;
                            const bool vc = valid(c);
#pragma unroll
                            for (int h = 0; h < 8; ++h) {
                                const int rl = rb + 16 * h, row = r0 + rl;
                                float2 x = make_float2(0.f, 0.f);
                                if (vc && row < m) x = Xs[(size_t)c * m + row];
                                st_split(ah, al, sw128_off(rl, c), kt ? x.y : x.x);
                            }
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncthreads();
                        if (tid == 0) {
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t ah = sbase + OFF_T, al = ah + TILE128;
                            const uint32_t bh = sbase + OFF_B + kt * 2 * TILE64, bl = bh + TILE64;
                            mma_ktile(t_upd, ah, al, bh, bl, idesc, kt == 0);
                            mma_commit(bar0);
                            pend[0] = true;
                            s_ok = wait_bar(0, lim);   // the next A tile reuses the buffer
                        }
                        __syncthreads();
                        if (!s_ok) {
                            fail = true;
                            break;
                        }
                    }
                    if (fail) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    {
                        // every warp: lanes of its TMEM quarter (rows), 8 of the 32 columns
                        const int qtr = warp & 3, cg = warp >> 2;
                        const int row = r0 + qtr * 32 + lane;
                        const uint32_t lane_off = (uint32_t)(qtr * 32) << 16;
                        float cr[8], ci[8];
                        tmem_ld8(t_upd + lane_off + 8 * cg, cr);
                        tmem_ld8(t_upd + lane_off + GC + 8 * cg, ci);
                        if (row < m) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int c = 8 * cg + e;
                                if (!valid(c)) continue;
                                const int gc = c < GB ? colI + c : colJ + c - GB;
                                const float2 x = Xs[(size_t)c * m + row];
                                __stcg(Wm + (size_t)gc * m + row, make_float2(x.x + cr[e], x.y + ci[e]));
                            }
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncthreads();
                }
            }
        }
        if (fail) {
            // drain what is still in flight, then leave with the gate unfinished
            if (tid == 0) {
                wait_bar(0, kGramSpin);
                wait_bar(1, kGramSpin);
                out->status = 5;
                atomicExch(&ctl->error, 1);
                s_fail = 1;
            }
            __syncthreads();
            break;
        }
        __threadfence();   // every thread's column stores before the report
        __syncthreads();
        if (tid == 0) {
            if (s_rot) {
                atomicAdd(&out->rot_sweep, s_rot);
                atomicAdd(&out->rotations, (unsigned long long)s_rot);
            }
            if (s_vis) atomicAdd(&out->visits, (unsigned long long)s_vis);
            __threadfence();
            const int dn = atomicAdd(&out->done, 1) + 1;
            if (dn == tgr.V) {
                out->done = 0;
                bool fin = false;
                if (round == R - 1) {
                    const int rs = atomicExch(&out->rot_sweep, 0);
                    if (rs == 0 || sweep + 1 >= max_sweeps) {
                        fin = true;
                        out->sweeps = sweep + 1;
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(256));
}

// Launch: one CTA of 512 threads per SM (about 222 KB of shared memory); no more CTAs
// than visits of a round can use.  Gates of more than 512 rows take the column kernel.
cudaError_t launch_jacobi_tc(const GateDesc* d, int n_gates, int n_lead, int n_max, double tol, int max_sweeps,
                             JacobiCtl* ctl, cudaStream_t s, unsigned spin_limit) {
    if (n_gates <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_jacobi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_tc, GT, SMEM_BYTES)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int nb = (n_max + GB - 1) / GB;
    const long long visits = (long long)n_gates * ((nb == 1) ? 1 : (nb + (nb & 1)) / 2);
    long long grid = (long long)sms;   // one CTA per SM: each holds 128 TMEM columns and most of the shared memory
    if (grid > visits) grid = visits;
    if (grid < 1) grid = 1;
    const int lead = (n_lead < 1 || n_lead > n_gates) ? n_gates : n_lead;
    k_jacobi_tc<<<(unsigned)grid, GT, SMEM_BYTES, s>>>(d, n_gates, lead, tol, max_sweeps < 1 ? 1 : max_sweeps, ctl,
                                                       spin_limit ? spin_limit : kSpinLimit);
    return cudaGetLastError();
}

int jacobi_tc_max_rows() { return GM; }

}  // namespace tnsim
