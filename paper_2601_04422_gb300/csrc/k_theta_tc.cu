// Tensor-core (tcgen05) merge + gate kernel for complex64 states.
//
// theta = G' . (A . B) as in k_gemm.cu (Fig. 2, Eq. 1), with the complex GEMM run on
// the 5th-generation tensor cores as real GEMMs on split operands:
//
//   1. k_split writes, for every gate, K-major planes of its two sites:
//        A (rows (l, p0), K = chi_M)            -> A_re_hi, A_re_lo, A_im_hi, A_im_lo
//        B^T (rows (p1, r), K = chi_M, transposed) -> B_re_hi, B_re_lo, B_im_hi, B_im_lo
//      where x = hi + lo, hi = x rounded to the tensor-core input type (TF32 or BF16)
//      and lo = (x - hi) rounded again ("3xTF32" / "BF16x3" splitting).  K is padded
//      with zeros to a multiple of the shared-memory stage.
//   2. k_theta_tc: one CTA (4 warps) per 128 x 128 output tile.  The tile's rows are
//      64 values of l (both p0), its columns 64 values of r for p1 = 0 and the same 64
//      for p1 = 1, so the gate mix of Eq. 1 stays inside the tile.  Per K stage the
//      eight plane tiles arrive by TMA (128-byte swizzle) on an mbarrier, then one
//      thread issues, per 8 (TF32) or 16 (BF16) K values, twelve tcgen05.mma into two
//      TMEM accumulators:
//        Re += Ar.Br - Ai.Bi,  Im += Ar.Bi + Ai.Br,   X.Y ~ Xhi.Yhi + Xhi.Ylo + Xlo.Yhi
//      (the minus via the instruction's negate-A bit).  The epilogue reads TMEM with
//      tcgen05.ld (thread = row), exchanges the partner row (l, 1 - p0) by shuffle,
//      applies the 4x4 gate in registers and writes theta column-major into W and
//      theta0, accumulating |theta|_F^2 in FP64.
// Every wait on an mbarrier is bounded (GateDesc::wait_polls polls, default 2^26).  On
// timeout the CTA stops issuing work, waits (again bounded, with the default limit)
// for the one barrier phase still pending -- the TMA copies or the MMAs it issued --
// so that nothing it started still writes its shared memory or its TMEM, then sets
// the gate's status to 5 (reported as ETIMEOUT), releases its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_common.cuh"
#include "tnsim_internal.h"

namespace tnsim {

constexpr int TC_M = 128;          // output tile rows (64 l x 2 p0)
constexpr int TC_RH = 64;          // r values per tile (two halves: p1 = 0, 1)
constexpr int TC_N = 2 * TC_RH;    // output tile columns
constexpr int TC_THREADS = 128;
constexpr unsigned kTcSpin = 1u << 26;     // default polls of a bounded mbarrier wait (about a second)

// ---------------------------------------------------------------- split pass

template <int MODE>  // 0: TF32 (planes of fp32 words), 1: BF16
struct PlaneT;
template <> struct PlaneT<0> { typedef float type; static constexpr int KS = 32; };
template <> struct PlaneT<1> { typedef __nv_bfloat16 type; static constexpr int KS = 64; };

template <int MODE>
__device__ __forceinline__ void split_store(typename PlaneT<MODE>::type* hi, typename PlaneT<MODE>::type* lo,
                                            size_t i, float v) {
    if constexpr (MODE == 0) {
        const float h = tf32_round(v);
        hi[i] = h;
        lo[i] = tf32_round(v - h);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// grid (row tiles of 32, k tiles of 32, gates * 2): z even = A planes, z odd = B^T planes
template <int MODE>
__global__ void __launch_bounds__(256) k_split(const GateDesc* __restrict__ gd) {
    typedef typename PlaneT<MODE>::type E;
    constexpr int KS = PlaneT<MODE>::KS;
    const GateDesc& d = gd[blockIdx.z >> 1];
    const bool isB = blockIdx.z & 1;
    const int q = d.q;
    const int chiL = d.chi[q], chiM = d.chi[q + 1], chiR = d.chi[q + 2];
    const int rows = isB ? 2 * chiR : 2 * chiL;
    const int kuse = (chiM + KS - 1) / KS * KS;
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    if (r0 >= rows || k0 >= kuse) return;
    const int RM = d.tc_rows, KM = d.tc_k;             // plane row count and K stride
    E* base = reinterpret_cast<E*>(d.tc_planes) + ((size_t)d.tc_slot * 8 + (isB ? 4 : 0)) * RM * KM;
    E* p_rh = base;
    E* p_rl = base + (size_t)RM * KM;
    E* p_ih = base + (size_t)2 * RM * KM;
    E* p_il = base + (size_t)3 * RM * KM;
    const float2* A = (const float2*)d.siteA;
    const float2* B = (const float2*)d.siteB;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (!isB) {
        // A rows (l, p0) are contiguous in k: read and write along k
        for (int rr = ty; rr < 32; rr += 8) {
            const int row = r0 + rr, k = k0 + tx;
            if (row >= rows) continue;
            float2 v = make_float2(0.f, 0.f);
            if (k < chiM) v = A[(size_t)row * chiM + k];
            const size_t i = (size_t)row * KM + k;
            split_store<MODE>(p_rh, p_rl, i, v.x);
            split_store<MODE>(p_ih, p_il, i, v.y);
        }
    } else {
        // B^T[n][k] = B[k][n] (n = p1 chi_R + r): transpose through shared memory
        __shared__ float2 t[32][33];
        const int n2 = 2 * chiR;
        for (int kk = ty; kk < 32; kk += 8) {
            const int k = k0 + kk, n = r0 + tx;
            float2 v = make_float2(0.f, 0.f);
            if (k < chiM && n < n2) v = B[(size_t)k * n2 + n];
            t[kk][tx] = v;
        }
        __syncthreads();
        for (int nn = ty; nn < 32; nn += 8) {
            const int n = r0 + nn, k = k0 + tx;
            if (n >= n2 || k >= kuse) continue;
            const float2 v = t[tx][nn];
            const size_t i = (size_t)n * KM + k;
            split_store<MODE>(p_rh, p_rl, i, v.x);
            split_store<MODE>(p_ih, p_il, i, v.y);
        }
    }
}

// ---------------------------------------------------------------- tcgen05 GEMM

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Instruction descriptor of this kernel's 128 x 128 tiles.
__device__ __forceinline__ uint32_t inst_desc(uint32_t fmt, uint32_t negA) { return idesc_mn(fmt, negA, TC_M, TC_N); }

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_theta_tc(const GateDesc* __restrict__ gd) {
    constexpr int KS = PlaneT<MODE>::KS;                    // K per stage (128 bytes)
    constexpr int KMMA = (MODE == 0) ? 8 : 16;               // K per MMA instruction
    constexpr uint32_t FMT = (MODE == 0) ? 2u : 1u;          // TF32 / BF16
    constexpr uint32_t TILE = TC_M * 128;                    // bytes of one 128-row plane tile
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q;
    const int chiL = d.chi[q], chiM = d.chi[q + 1], chiR = d.chi[q + 2];
    const int m = 2 * chiL;
    const int m0 = blockIdx.x * TC_M, r0 = blockIdx.y * TC_RH;
    if (m0 >= m || r0 >= chiR) return;
    const int kuse = (chiM + KS - 1) / KS * KS;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned: 4 A plane tiles then 4 B plane tiles (each 16 KB)
    unsigned char* tiles = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_full, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float2 Gs[16];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 16) {
        const int o = tid >> 2, i = tid & 3;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 4; ++j) {
            const double gr = d.g4[2 * (o * 4 + j)], gi = d.g4[2 * (o * 4 + j) + 1];
            double kr = (j == i) ? 1.0 : 0.0, ki = 0.0;
            if (d.uL || d.uR) {
                double ar = ((j >> 1) == (i >> 1)) ? 1.0 : 0.0, ai = 0.0;
                double br = ((j & 1) == (i & 1)) ? 1.0 : 0.0, bi = 0.0;
                if (d.uL) { ar = d.uL[2 * ((j >> 1) * 2 + (i >> 1))]; ai = d.uL[2 * ((j >> 1) * 2 + (i >> 1)) + 1]; }
                if (d.uR) { br = d.uR[2 * ((j & 1) * 2 + (i & 1))]; bi = d.uR[2 * ((j & 1) * 2 + (i & 1)) + 1]; }
                kr = ar * br - ai * bi;
                ki = ar * bi + ai * br;
            }
            re += gr * kr - gi * ki;
            im += gr * ki + gi * kr;
        }
        Gs[tid] = make_float2((float)re, (float)im);
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bar_full), 1);
        mbar_init(smem_u32(&bar_mma), 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t t_re = tmem_base, t_im = tmem_base + TC_N;

    const CUtensorMap* mapA = reinterpret_cast<const CUtensorMap*>(d.tc_map_a);
    const CUtensorMap* mapB = reinterpret_cast<const CUtensorMap*>(d.tc_map_b);
    const int zA = d.tc_slot * 8, zB = d.tc_slot * 8 + 4;
    const uint32_t sbase = smem_u32(tiles);
    const int nk = kuse / KS;
    const unsigned lim = d.wait_polls > 0 ? (unsigned)d.wait_polls : kTcSpin;
    uint32_t pend_bar = 0, pend_phase = 0;   // the barrier phase left pending by a timeout
    for (int kb = 0; kb < nk; ++kb) {
        if (tid == 0 && !s_fail) {
            mbar_expect_tx(smem_u32(&bar_full), 8 * TILE);
            for (int p = 0; p < 4; ++p) tma_load_3d(sbase + p * TILE, mapA, kb * KS, m0, zA + p, smem_u32(&bar_full));
            for (int p = 0; p < 4; ++p) {
                tma_load_3d(sbase + (4 + p) * TILE, mapB, kb * KS, r0, zB + p, smem_u32(&bar_full));
                tma_load_3d(sbase + (4 + p) * TILE + TILE / 2, mapB, kb * KS, chiR + r0, zB + p, smem_u32(&bar_full));
            }
        }
        if (!mbar_wait(smem_u32(&bar_full), kb & 1, lim)) atomicExch(&s_fail, 1);
        __syncthreads();
        if (s_fail) {
            // the copies of this stage may still be in flight (no MMA of it was issued)
            pend_bar = smem_u32(&bar_full);
            pend_phase = kb & 1;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // plane tiles: 0 A_re_hi, 1 A_re_lo, 2 A_im_hi, 3 A_im_lo, 4 B_re_hi, 5 B_re_lo, 6 B_im_hi, 7 B_im_lo
            const uint32_t idp = inst_desc(FMT, 0), idn = inst_desc(FMT, 1);
            for (int j = 0; j < KS / KMMA; ++j) {
                const uint32_t off = j * KMMA * (MODE == 0 ? 4 : 2);
                uint64_t a[4], b[4];
                for (int p = 0; p < 4; ++p) {
                    a[p] = smem_desc(sbase + p * TILE + off);
                    b[p] = smem_desc(sbase + (4 + p) * TILE + off);
                }
                const uint32_t acc0 = (kb > 0 || j > 0) ? 1u : 0u;
                // Re += Ar Br - Ai Bi  (hi.hi + hi.lo + lo.hi)
                mma<MODE>(t_re, a[0], b[0], idp, acc0);
                mma<MODE>(t_re, a[0], b[1], idp, 1u);
                mma<MODE>(t_re, a[1], b[0], idp, 1u);
                mma<MODE>(t_re, a[2], b[2], idn, 1u);
                mma<MODE>(t_re, a[2], b[3], idn, 1u);
                mma<MODE>(t_re, a[3], b[2], idn, 1u);
                // Im += Ar Bi + Ai Br
                mma<MODE>(t_im, a[0], b[2], idp, acc0);
                mma<MODE>(t_im, a[0], b[3], idp, 1u);
                mma<MODE>(t_im, a[1], b[2], idp, 1u);
                mma<MODE>(t_im, a[2], b[0], idp, 1u);
                mma<MODE>(t_im, a[2], b[1], idp, 1u);
                mma<MODE>(t_im, a[3], b[0], idp, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_mma))
                         : "memory");
        }
        // the stage buffers are reused by the next TMA only after the MMAs read them
        if (!mbar_wait(smem_u32(&bar_mma), kb & 1, lim)) atomicExch(&s_fail, 1);
        __syncthreads();
        if (s_fail) {
            // this stage's copies have landed; its MMAs may still be running
            pend_bar = smem_u32(&bar_mma);
            pend_phase = kb & 1;
            break;
        }
    }
    if (s_fail && tid == 0) mbar_wait(pend_bar, pend_phase, kTcSpin);   // drain before TMEM and smem go
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!s_fail) {
        // epilogue: thread = tile row (TMEM lane), warp w owns lanes 32w..32w+31
        float2* Wm = (float2*)d.W;
        float2* T0 = (float2*)d.theta0;
        const int i_t = warp * 32 + lane;
        const int row = m0 + i_t;          // (l, c) = (row / 2, row % 2)
        const int c = row & 1;
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        SqAcc<float> fsq;  // |theta|_F^2 of this thread's elements
        for (int rc = 0; rc < TC_RH; rc += 16) {
            float re0[16], im0[16], re1[16], im1[16];
            tmem_ld16(t_re + lane_off + rc, re0);
            tmem_ld16(t_im + lane_off + rc, im0);
            tmem_ld16(t_re + lane_off + TC_RH + rc, re1);
            tmem_ld16(t_im + lane_off + TC_RH + rc, im1);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                // M[(l, c)][(d, r)] for both d, own row c and the partner row 1 - c
                float2 mo[2] = {make_float2(re0[e], im0[e]), make_float2(re1[e], im1[e])};
                float2 mp[2];
                mp[0].x = __shfl_xor_sync(0xffffffffu, mo[0].x, 1);
                mp[0].y = __shfl_xor_sync(0xffffffffu, mo[0].y, 1);
                mp[1].x = __shfl_xor_sync(0xffffffffu, mo[1].x, 1);
                mp[1].y = __shfl_xor_sync(0xffffffffu, mo[1].y, 1);
                const int r = r0 + rc + e;
                if (row < m && r < chiR) {
#pragma unroll
                    for (int bb = 0; bb < 2; ++bb) {
                        float2 t = make_float2(0.f, 0.f);
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                            for (int dd = 0; dd < 2; ++dd) {
                                const float2 g = Gs[(2 * c + bb) * 4 + 2 * cc + dd];
                                const float2 v = (cc == c) ? mo[dd] : mp[dd];
                                t.x = fmaf(g.x, v.x, fmaf(-g.y, v.y, t.x));
                                t.y = fmaf(g.x, v.y, fmaf(g.y, v.x, t.y));
                            }
                        const size_t idx = (size_t)(bb * chiR + r) * m + row;
                        Wm[idx] = t;
                        T0[idx] = t;
                        fsq.add(t.x);
                        fsq.add(t.y);
                    }
                }
            }
        }
        double fro = fsq.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
        if (lane == 0 && fro != 0.0) atomicAdd(&d.out->frob2, fro);
    } else if (tid == 0) {
        d.out->status = 5;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * TC_N));
    }
}

template <int MODE>
static cudaError_t launch_tc(const GateDesc* d, int n_gates, int chiL_max, int chiR_max, int kmax, cudaStream_t s) {
    constexpr int KS = PlaneT<MODE>::KS;
    dim3 gs((2 * max(chiL_max, chiR_max) + 31) / 32, (kmax + KS - 1) / KS * KS / 32, 2 * n_gates);
    k_split<MODE><<<gs, 256, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = 8 * TC_M * 128 + 1024;
    e = cudaFuncSetAttribute(k_theta_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((2 * chiL_max + TC_M - 1) / TC_M, (chiR_max + TC_RH - 1) / TC_RH, n_gates);
    k_theta_tc<MODE><<<grid, TC_THREADS, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_theta_tc(int mode, const GateDesc* d, int n_gates, int chiL_max, int chiM_max, int chiR_max,
                            cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    return mode == 0 ? launch_tc<0>(d, n_gates, chiL_max, chiR_max, chiM_max, s)
                     : launch_tc<1>(d, n_gates, chiL_max, chiR_max, chiM_max, s);
}

// ---------------------------------------------------------------- tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Encode the A-box (128 rows) and B-box (64 rows) maps over a plane buffer laid out as
// [slots * 8][rows][kstride] of fp32 (mode 0) or bf16 (mode 1) elements.
cudaError_t encode_plane_maps(int mode, void* planes, int slots, int rows, int kstride, CUtensorMap* host_a,
                              CUtensorMap* host_b) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
        fn = (EncodeTiledFn)p;
    }
    const size_t esz = mode == 0 ? 4 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)kstride, (cuuint64_t)rows, (cuuint64_t)slots * 8};
    const cuuint64_t strides[2] = {(cuuint64_t)kstride * esz, (cuuint64_t)rows * kstride * esz};
    const cuuint32_t kbox = (cuuint32_t)(128 / esz);
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint32_t boxA[3] = {kbox, (cuuint32_t)TC_M, 1};
    const cuuint32_t boxB[3] = {kbox, (cuuint32_t)TC_RH, 1};
    CUresult r = fn(host_a, dt, 3, planes, dims, strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = fn(host_b, dt, 3, planes, dims, strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace tnsim
