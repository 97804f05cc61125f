// Scheduling and rotation-parameter pieces shared by the two persistent Jacobi
// kernels (k_jacobi.cu: rotations on the columns; k_jacobi_tc.cu: rotations on the
// block pair's Gram matrix with tensor-core block products).
#pragma once
#include <float.h>

#include "tnsim_internal.h"

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

// Rotation parameters (c - 1, s e^{i phi}) of a column pair from a, b and g = gr + i gi.
// The quantities that decide whether the rotation is unitary -- |e^{i phi}| = 1 and
// c^2 + s^2 = 1 -- use correctly rounded square roots and reciprocals (sqrtf,
// __frcp_rn), so their rounding errors are unbiased; the skip test and the angle t
// (which only has to orthogonalise the pair to within rounding) use fast division.
// c - 1 = -t^2 / (rr (1 + rr)) is formed without cancellation.  FP64 keeps IEEE
// operations throughout.
__device__ __forceinline__ bool rot_params_fast(float a, float b, float gr, float gi, float tol2, float zthr,
                                                float& cm1, float& sr, float& si, float& tg) {
    const float g2 = gr * gr + gi * gi;
    if (!(a > zthr && b > zthr && __fdividef(g2, b) > tol2 * a)) return false;
    const float gabs = sqrtf(g2);
    const float rg = __frcp_rn(gabs);                     // 1 / |g|
    const float zeta = 0.5f * (b - a) * rg;
    const float az = fabsf(zeta);
    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); for |zeta| > 2^12, 1 + zeta^2 rounds to zeta^2
    const float den = az > 4096.f ? 2.f * az : az + sqrtf(fmaf(zeta, zeta, 1.f));
    const float t = copysignf(__fdividef(1.f, den), zeta);
    const float rr = sqrtf(fmaf(t, t, 1.f));
    const float irr = __frcp_rn(rr);                      // c
    cm1 = -(t * t) * irr * __frcp_rn(1.f + rr);
    const float sv = t * irr;
    sr = sv * (gr * rg);
    si = sv * (gi * rg);
    tg = t * gabs;                                        // the norms become a - t|g|, b + t|g|
    return true;
}
__device__ __forceinline__ bool rot_params_fast(double a, double b, double gr, double gi, double tol2, double zthr,
                                                double& cm1, double& sr, double& si, double& tg) {
    const double g2 = gr * gr + gi * gi;
    if (!(a > zthr && b > zthr && g2 / b > tol2 * a)) return false;
    const double gabs = sqrt(g2);
    const double zeta = (b - a) / (2 * gabs);
    const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    const double rr = sqrt(1.0 + t * t);
    cm1 = -(t * t) / (rr * (1.0 + rr));
    const double sv = t / rr;
    sr = sv * (gr / gabs);
    si = sv * (gi / gabs);
    tg = t * gabs;
    return true;
}

// Geometry of one gate's tournament: nb column blocks, P players (nb rounded up to
// even), R rounds per sweep and V visits (block pairs) per round.
struct Tour {
    int m, n, nb, P, R, V;
};
template <int BC>
__device__ __forceinline__ Tour tour_of(const GateDesc& d) {
    Tour t;
    t.m = 2 * d.chi[d.q];
    t.n = 2 * d.chi[d.q + 2];
    t.nb = (t.n + BC - 1) / BC;
    t.P = t.nb + (t.nb & 1);
    t.R = (t.nb == 1) ? 1 : t.P - 1;
    t.V = (t.nb == 1) ? 1 : t.P / 2;
    return t;
}

constexpr unsigned kSpinLimit = 1u << 22;   // default idle polls without any progress before giving up
constexpr int kScanTable = 2048;              // gates whose visit count is cached in shared memory

// Warp-parallel claim of one visit (warp 0): each lane checks one gate per pass (one
// L2 round trip), the first claimable gate in descriptor order from gate scan0 on
// (wrapping around) is tried with an atomic.  found = 0 when nothing is claimable now.
template <int BC>
__device__ __forceinline__ void claim_scan(const GateDesc* __restrict__ gd, int n_gates, const short* s_V, int scan0,
                                           int lane, int& found, int& fg, int& frnd, int& fv) {
    found = 0;
    fg = -1;
    frnd = 0;
    fv = 0;
    const int nchunks = (n_gates + 31) / 32;
    for (int c = 0; c < nchunks && !found; ++c) {
        const int k = 32 * c + lane;
        const int g = k < n_gates ? (scan0 + k) % n_gates : n_gates;   // every gate once
        bool ok = false;
        int V = 0;
        GateOut* o = nullptr;
        if (g < n_gates) {
            o = gd[g].out;
            V = g < kScanTable ? (int)s_V[g] : tour_of<BC>(gd[g]).V;
            const int fin = *((volatile int*)&o->finished);
            const unsigned long long cur = *((volatile unsigned long long*)&o->claim);
            ok = !fin && (unsigned)(cur & 0xffffffffull) < (unsigned)V;
        }
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        while (mask && !found) {
            const int l = __ffs(mask) - 1;
            int got = 0;
            if (lane == l) {
                const unsigned long long st = atomicAdd(&o->claim, 1ull);
                if ((unsigned)(st & 0xffffffffull) < (unsigned)V) {
                    got = 1;
                    fg = g;
                    frnd = (int)(st >> 32);
                    fv = (int)(st & 0xffffffffull);
                }
            }
            got = __shfl_sync(0xffffffffu, got, l);
            if (got) {
                fg = __shfl_sync(0xffffffffu, fg, l);
                frnd = __shfl_sync(0xffffffffu, frnd, l);
                fv = __shfl_sync(0xffffffffu, fv, l);
                found = 1;
            }
            mask &= mask - 1;
        }
    }
}

// Both blocks of a visit into shared memory with asynchronous 16-byte copies
// (cp.async.cg: through L2, no registers held), so every copy of both blocks is in
// flight at once; the caller's barrier follows the wait.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
template <typename C>
__device__ __forceinline__ void copy_blocks_in(C* dI, const C* sI, int countI, C* dJ, const C* sJ, int countJ) {
    const int uI = (int)((size_t)countI * sizeof(C) / 16), uJ = (int)((size_t)countJ * sizeof(C) / 16);
    const int4* a = reinterpret_cast<const int4*>(sI);
    const int4* b = reinterpret_cast<const int4*>(sJ);
    int4* da = reinterpret_cast<int4*>(dI);
    int4* db = reinterpret_cast<int4*>(dJ);
    for (int i = threadIdx.x; i < uI; i += blockDim.x) cp_async16(da + i, a + i);
    for (int i = threadIdx.x; i < uJ; i += blockDim.x) cp_async16(db + i, b + i);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
}  // namespace tnsim
