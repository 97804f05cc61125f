// Left site of a QR-preconditioned complex64 gate on the tcgen05 tensor cores.
//
// With the Jacobi iteration run on R^H (k_qr.cu), the converged columns W' = U'' S give
// the left site as one product, U = theta V S^-1 = theta W'_k S^-2 (Sec. IV.A: the site
// that keeps U): an (m x n) . (n x k) complex product, theta0 column-major and the kept
// columns perm[j] of W' scaled by 1 / s_j^2.  Here it runs as real products on split
// operands (3xTF32: x = hi + lo, hi.hi + hi.lo + lo.hi, FP32 accumulation in TMEM), four
// real products per complex one (Re += Ar Br - Ai Bi, Im += Ar Bi + Ai Br, the minus by
// the instruction's negate-A bit).  One CTA computes a 128 x 256 tile of U (an M = 128,
// K = 8 TF32 MMA costs the same at any N up to 256 on this GPU, so N = 256 is the
// cheapest per output element).  Per K chunk of 32 the 512 threads write the split
// operand tiles (128-byte-swizzled K-major) into shared memory, one thread issues the
// 48 MMAs, and their completion is awaited on an mbarrier with a bounded wait (on
// timeout the gate reports status 5).
#include "tc_common.cuh"
#include "tnsim_internal.h"

namespace tnsim {

namespace {

constexpr int LP_M = 128;                  // rows of U per CTA
constexpr int LP_N = 256;                  // kept columns per CTA
constexpr int LP_T = 512;                  // threads
constexpr uint32_t LP_AT = LP_M * 128;     // bytes of one A plane tile (32 K values per row)
constexpr uint32_t LP_BT = LP_N * 128;     // bytes of one B plane tile
constexpr uint32_t LP_SMEM = 4 * LP_AT + 4 * LP_BT + 1024;
constexpr unsigned kLpSpin = 1u << 26;

__device__ __forceinline__ void lp_split(unsigned char* base, uint32_t tile, uint32_t off, float2 v) {
    // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
    const float rh = tf32_round(v.x), ih = tf32_round(v.y);
    *reinterpret_cast<float*>(base + 0 * tile + off) = rh;
    *reinterpret_cast<float*>(base + 1 * tile + off) = tf32_round(v.x - rh);
    *reinterpret_cast<float*>(base + 2 * tile + off) = ih;
    *reinterpret_cast<float*>(base + 3 * tile + off) = tf32_round(v.y - ih);
}

}  // namespace

__global__ void __launch_bounds__(LP_T, 1) k_left_pre_tc(const GateDesc* __restrict__ gd) {
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q, m = 2 * d.chi[q], n = 2 * d.chi[q + 2];
    if (!qr_active(d, m, n)) return;
    const int k = d.out->k;
    const int r0 = blockIdx.x * LP_M, j0 = blockIdx.y * LP_N;
    if (r0 >= m || j0 >= k) return;   // uniform over the CTA, before any TMEM is held
    extern __shared__ unsigned char lp_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)lp_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* At = sm;                    // 4 A planes
    unsigned char* Bt = sm + 4 * LP_AT;        // 4 B planes
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    __shared__ int pj[LP_N];
    __shared__ float fj[LP_N];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int j = tid; j < LP_N; j += LP_T) {
        const int jj = j0 + j;
        pj[j] = jj < k ? d.perm[jj] : -1;
        const double s2 = jj < k ? d.s2[jj] : 0.0;
        fj[j] = s2 > 0.0 ? (float)(1.0 / s2) : 0.f;
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * LP_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t t_re = tmem_base, t_im = tmem_base + LP_N;
    const uint32_t id_p = idesc_mn(2u, 0u, LP_M, LP_N), id_n = idesc_mn(2u, 1u, LP_M, LP_N);
    const uint32_t sa = smem_u32(At), sb = smem_u32(Bt);
    const unsigned lim = d.wait_polls > 0 ? (unsigned)d.wait_polls : kLpSpin;
    const float2* T0 = (const float2*)d.theta0;
    const float2* W = (const float2*)d.W;
    uint32_t phase = 0;
    bool fail = false;
    // Operands of a K chunk, held in registers so that the next chunk's loads overlap the
    // current chunk's MMAs.  A: lane = K index, warp = 8 rows (a warp's stores then fill
    // one 128-byte tile row: no bank conflicts; its loads are 32 runs of 64 bytes).  B:
    // lane = K index, warp = 16 kept columns (coalesced 256-byte loads).
    float4 ra[4];
    float2 rb[16];
    auto load_chunk = [&](int kc) {
        const int kk = lane, rr = warp * 8;
        const bool kin = kc + kk < n;
        const float2* srca = T0 + (size_t)(kc + kk) * m + r0 + rr;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            ra[h] = (kin && r0 + rr + 2 * h < m) ? __ldcg(reinterpret_cast<const float4*>(srca + 2 * h))
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int h = 0; h < 16; ++h) {
            const int pc = pj[warp * 16 + h];
            rb[h] = (pc >= 0 && kin) ? __ldcg(W + (size_t)pc * n + kc + kk) : make_float2(0.f, 0.f);
        }
    };
    load_chunk(0);
    for (int kc = 0; kc < n; kc += 32) {
        if (kc > 0) {
            // the previous chunk's MMAs must have read the tiles before they are rewritten
            if (tid == 0) {
                s_ok = mbar_wait(smem_u32(&bar), phase, lim);
                if (!s_ok) mbar_wait(smem_u32(&bar), phase, kLpSpin);   // drain before leaving
            }
            __syncthreads();
            phase ^= 1u;
            if (!s_ok) {
                fail = true;
                break;
            }
        }
        {
            const int kk = lane, rr = warp * 8;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                lp_split(At, LP_AT, sw128_off(rr + 2 * h, kk), make_float2(ra[h].x, ra[h].y));
                lp_split(At, LP_AT, sw128_off(rr + 2 * h + 1, kk), make_float2(ra[h].z, ra[h].w));
            }
#pragma unroll
            for (int h = 0; h < 16; ++h) {
                const int j = warp * 16 + h;
                const float f = fj[j];
                lp_split(Bt, LP_BT, sw128_off(j, kk), make_float2(rb[h].x * f, rb[h].y * f));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint64_t a[4], b[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    a[p] = smem_desc(sa + p * LP_AT + 32 * j);
                    b[p] = smem_desc(sb + p * LP_BT + 32 * j);
                }
                const uint32_t acc0 = (kc > 0 || j > 0) ? 1u : 0u;
                // Re += Ar Br - Ai Bi (hi.hi + hi.lo + lo.hi)
                mma_tf32(t_re, a[0], b[0], id_p, acc0);
                mma_tf32(t_re, a[0], b[1], id_p, 1u);
                mma_tf32(t_re, a[1], b[0], id_p, 1u);
                mma_tf32(t_re, a[2], b[2], id_n, 1u);
                mma_tf32(t_re, a[2], b[3], id_n, 1u);
                mma_tf32(t_re, a[3], b[2], id_n, 1u);
                // Im += Ar Bi + Ai Br
                mma_tf32(t_im, a[0], b[2], id_p, acc0);
                mma_tf32(t_im, a[0], b[3], id_p, 1u);
                mma_tf32(t_im, a[1], b[2], id_p, 1u);
                mma_tf32(t_im, a[2], b[0], id_p, 1u);
                mma_tf32(t_im, a[2], b[1], id_p, 1u);
                mma_tf32(t_im, a[3], b[0], id_p, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
        }
        if (kc + 32 < n) load_chunk(kc + 32);   // in flight while the MMAs run
    }
    if (!fail) {
        if (tid == 0) {
            s_ok = mbar_wait(smem_u32(&bar), phase, lim);
            if (!s_ok) mbar_wait(smem_u32(&bar), phase, kLpSpin);
        }
        __syncthreads();
        fail = !s_ok;
    }
    if (!fail) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // every warp: the rows of its TMEM quarter, 64 of the 256 columns
        const int qtr = warp & 3, cg = warp >> 2;
        const int r = r0 + qtr * 32 + lane;
        const uint32_t lane_off = (uint32_t)(qtr * 32) << 16;
        float2* U = (float2*)d.siteA;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float re[16], im[16];
            tmem_ld16(t_re + lane_off + 64 * cg + c0, re);
            tmem_ld16(t_im + lane_off + 64 * cg + c0, im);
            const int jb = j0 + 64 * cg + c0;
            if (r < m) {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    if (jb + e < k) U[(size_t)r * k + jb + e] = make_float2(re[e], im[e]);
            }
        }
    } else if (tid == 0) {
        d.out->status = 5;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * LP_N));
}

cudaError_t launch_left_pre_tc(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_left_pre_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP_SMEM);
    if (e != cudaSuccess) return e;
    dim3 g((m_max + LP_M - 1) / LP_M, (k_max + LP_N - 1) / LP_N, n_gates);
    k_left_pre_tc<<<g, LP_T, LP_SMEM, s>>>(d);
    return cudaGetLastError();
}

}  // namespace tnsim
