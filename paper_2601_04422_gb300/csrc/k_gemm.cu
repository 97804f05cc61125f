// Contractions of the two-qubit update.
//
//  k_theta : merge of the two sites over their shared bond (Fig. 2) fused with the
//            4x4 gate contraction (Eq. 1).  Viewed as matrices, site q is
//            A = (2chi_L) x chi_M with rows (l, p0) and site q+1 is
//            B = chi_M x (2chi_R) with columns (p1, r), so the merge is one complex
//            GEMM M = A.B.  The gate only mixes the 2x2 block
//            {rows (l,0),(l,1)} x {columns (0,r),(1,r)} of M, so every thread owns
//            complete blocks and applies the gate in registers before the store.
//            theta is written column-major (the layout the one-sided Jacobi SVD
//            orthogonalises), twice: into the working matrix W and into theta0.
//  k_right : the new right site S.V^H (Sec. III.A "Two Qubit Gate").  With W = theta.V
//            and U = W.S^-1, row j of S.V^H equals u_j^H theta, so the right site is
//            the product U_kept^H . theta0 scaled per row -- no V is accumulated.
//            In canonical form (k_canon.cu) it is V^H of diag(Lam_q) theta instead.
#include "tnsim_internal.h"

namespace tnsim {

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfma_conj(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------
// K1: theta[(l,a),(b,r)] = sum_{c,d} G'[2a+b][2c+d] sum_m A[l,c,m] B[m,d,r]
// with G' = G . (uL (x) uR) when one-qubit gates precede the pair.
// CTA tile: 32 l x 32 r (all four (c,d) combinations), K step 16, 256 threads;
// thread (tx, ty) owns l in {tx, tx+16}, r in {ty, ty+16}.
constexpr int TH_L = 32, TH_R = 32, TH_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_theta(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q;
    const int chiL = d.chi[q], chiM = d.chi[q + 1], chiR = d.chi[q + 2];
    const int l0 = blockIdx.x * TH_L, r0 = blockIdx.y * TH_R;
    if (l0 >= chiL || r0 >= chiR) return;

    __shared__ __align__(16) C As[TH_K][2 * TH_L];   // [k][2*li + c]
    __shared__ __align__(16) C Bs[TH_K][2 * TH_R];   // [k][dd*32 + ri]
    __shared__ C Gs[16];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < 16) {
        const int o = tid >> 2, i = tid & 3;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 4; ++j) {
            double gr = d.g4[2 * (o * 4 + j)], gi = d.g4[2 * (o * 4 + j) + 1];
            // K[j][i] = uL[j>>1][i>>1] * uR[j&1][i&1]
            double kr = (j == i) ? 1.0 : 0.0, ki = 0.0;
            if (d.uL || d.uR) {
                double ar = ((j >> 1) == (i >> 1)) ? 1.0 : 0.0, ai = 0.0;
                double br = ((j & 1) == (i & 1)) ? 1.0 : 0.0, bi = 0.0;
                if (d.uL) { ar = d.uL[2 * ((j >> 1) * 2 + (i >> 1))]; ai = d.uL[2 * ((j >> 1) * 2 + (i >> 1)) + 1]; }
                if (d.uR) { br = d.uR[2 * ((j & 1) * 2 + (i & 1))]; bi = d.uR[2 * ((j & 1) * 2 + (i & 1)) + 1]; }
                kr = ar * br - ai * bi; ki = ar * bi + ai * br;
            }
            re += gr * kr - gi * ki; im += gr * ki + gi * kr;
        }
        Gs[tid].x = (T)re; Gs[tid].y = (T)im;
    }

    const C* A = (const C*)d.siteA;
    const C* B = (const C*)d.siteB;
    C acc[2][2][2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int e = 0; e < 2; ++e) { acc[i][j][c][e].x = 0; acc[i][j][c][e].y = 0; }

    const int a_row = tid >> 2, a_k = (tid & 3) * 4;          // A tile: 64 rows x 16 k
    const int b_k = tid >> 4, b_seg = tid & 15;               // B tile: 16 k x 64 cols
    const int b_dd = b_seg >> 3, b_r = (b_seg & 7) * 4;
    const int m = 2 * chiL;

    for (int k0 = 0; k0 < chiM; k0 += TH_K) {
        {
            const int grow = 2 * l0 + a_row;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + a_k + e;
                C v; v.x = 0; v.y = 0;
                if (grow < m && k < chiM) v = A[(size_t)grow * chiM + k];
                As[a_k + e][a_row] = v;
            }
            const int k = k0 + b_k;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = r0 + b_r + e;
                C v; v.x = 0; v.y = 0;
                if (k < chiM && r < chiR) v = B[((size_t)k * 2 + b_dd) * chiR + r];
                Bs[b_k][b_dd * TH_R + b_r + e] = v;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TH_K; ++kk) {
            C a[2][2], b[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                a[i][0] = As[kk][2 * (tx + 16 * i)];
                a[i][1] = As[kk][2 * (tx + 16 * i) + 1];
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                b[j][0] = Bs[kk][ty + 16 * j];
                b[j][1] = Bs[kk][TH_R + ty + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int e = 0; e < 2; ++e) cfma(acc[i][j][c][e], a[i][c], b[j][e]);
        }
        __syncthreads();
    }

    C* Wm = (C*)d.W;
    C* T0 = (C*)d.theta0;
    SqAcc<T> fsq;  // |theta|_F^2 of this thread's elements
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int l = l0 + tx + 16 * i;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + ty + 16 * j;
            if (l < chiL && r < chiR) {
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) {
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa) {
                        C t; t.x = 0; t.y = 0;
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int e = 0; e < 2; ++e)
                                cfma(t, Gs[(2 * aa + bb) * 4 + 2 * c + e], acc[i][j][c][e]);
                        const size_t idx = (size_t)(bb * chiR + r) * m + 2 * l + aa;
                        Wm[idx] = t;
                        T0[idx] = t;
                        fsq.add(t.x);
                        fsq.add(t.y);
                    }
                }
            }
        }
    }
    double fro = fsq.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0 && fro != 0.0) atomicAdd(&d.out->frob2, fro);
}

template <typename T>
cudaError_t launch_theta(const GateDesc* d, int n_gates, int chiL_max, int chiR_max,
                         cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    dim3 grid((chiL_max + TH_L - 1) / TH_L, (chiR_max + TH_R - 1) / TH_R, n_gates);
    k_theta<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4b: right site R[j, col] = f_j sum_row conj(W[row, perm_j]) theta0[row, col],
//      f_j = scale / s_{perm_j}; j < k, col < 2chi_R, row < 2chi_L.
// Output (k, 2, chi_R) row-major = R row-major with leading dimension 2chi_R.
// CTA tile 64 j x 64 col, K step 16 rows, 256 threads, 4x4 per thread.
constexpr int RT_J = 64, RT_C = 64, RT_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_right(const GateDesc* __restrict__ gd) {
    using C = typename CT<T>::type;
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q;
    const int chiL = d.chi[q], chiR = d.chi[q + 2];
    const int k = d.out->k;
    const int m = 2 * chiL, n = 2 * chiR;
    if (qr_active(d, m, n)) return;   // QR-preconditioned: k_right_pre (k_qr.cu)
    const int c0 = blockIdx.x * RT_C, j0 = blockIdx.y * RT_J;
    if (c0 >= n || j0 >= k) return;

    __shared__ __align__(16) C As[RT_K][RT_J];
    __shared__ __align__(16) C Bs[RT_K][RT_C];
    __shared__ int pj[RT_J];
    __shared__ T fj[RT_J];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < RT_J) {
        const int j = j0 + tid;
        if (j < k) {
            pj[tid] = d.perm[j];
            const double s2j = d.s2[j];
            // paper's form: row j of S.V^H (times the renormalisation); canonical form:
            // row j of V^H = u_j^H diag(Lam_q) theta / s_j = w_j^H diag(Lam_q) theta / s_j^2
            if (d.canon) fj[tid] = s2j > 0.0 ? (T)(1.0 / s2j) : (T)0;
            else fj[tid] = s2j > 0.0 ? (T)(d.out->scale / sqrt(s2j)) : (T)0;
        } else {
            pj[tid] = -1;
            fj[tid] = 0;
        }
    }
    __syncthreads();

    const C* Wm = (const C*)d.W;
    const C* T0 = (const C*)d.theta0;
    const int lk = d.canon ? *d.lam_k : 0;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j].x = 0; acc[i][j].y = 0; }

    const int ld_row = tid >> 2, ld_k = (tid & 3) * 4;
    for (int r0 = 0; r0 < m; r0 += RT_K) {
        {
            const int col_w = pj[ld_row];
            const int col_t = c0 + ld_row;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = r0 + ld_k + e;
                C v; v.x = 0; v.y = 0;
                if (col_w >= 0 && row < m) v = Wm[(size_t)col_w * m + row];
                As[ld_k + e][ld_row] = v;
                C w; w.x = 0; w.y = 0;
                if (col_t < n && row < m) w = T0[(size_t)col_t * m + row];
                if (d.canon && row < m && (row >> 1) < lk) {
                    const T f = (T)d.lam[row >> 1];
                    w.x *= f;
                    w.y *= f;
                }
                Bs[ld_k + e][ld_row] = w;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RT_K; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma_conj(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    C* R = (C*)d.siteB;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int jl = ty + 16 * i;
        const int j = j0 + jl;
        if (j >= k) continue;
        const T f = fj[jl];
#pragma unroll
        for (int jc = 0; jc < 4; ++jc) {
            const int col = c0 + tx + 16 * jc;
            if (col < n) {
                C v; v.x = acc[i][jc].x * f; v.y = acc[i][jc].y * f;
                R[(size_t)j * n + col] = v;
            }
        }
    }
}

template <typename T>
cudaError_t launch_right(const GateDesc* d, int n_gates, int k_max, int n_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    dim3 grid((n_max + RT_C - 1) / RT_C, (k_max + RT_J - 1) / RT_J, n_gates);
    k_right<T><<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K1 with three real products per complex product (FP32, SIMT): for a = ar + i ai and
// b = br + i bi, p1 = ar br, p2 = ai bi, p3 = (ar + ai)(br + bi), so
// Re(a b) = p1 - p2 and Im(a b) = p3 - p1 - p2; the sums ar + ai and br + bi are formed
// once per loaded element.  Same tiling and epilogue as k_theta.
__global__ void __launch_bounds__(256) k_theta_3m(const GateDesc* __restrict__ gd) {
    using C = float2;
    const GateDesc& d = gd[blockIdx.z];
    const int q = d.q;
    const int chiL = d.chi[q], chiM = d.chi[q + 1], chiR = d.chi[q + 2];
    const int l0 = blockIdx.x * TH_L, r0 = blockIdx.y * TH_R;
    if (l0 >= chiL || r0 >= chiR) return;
    __shared__ __align__(16) float3 As[TH_K][2 * TH_L];   // (re, im, re + im)
    __shared__ __align__(16) float3 Bs[TH_K][2 * TH_R];
    __shared__ C Gs[16];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < 16) {
        const int o = tid >> 2, i = tid & 3;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 4; ++j) {
            double gr = d.g4[2 * (o * 4 + j)], gi = d.g4[2 * (o * 4 + j) + 1];
            double kr = (j == i) ? 1.0 : 0.0, ki = 0.0;
            if (d.uL || d.uR) {
                double ar = ((j >> 1) == (i >> 1)) ? 1.0 : 0.0, ai = 0.0;
                double br = ((j & 1) == (i & 1)) ? 1.0 : 0.0, bi = 0.0;
                if (d.uL) { ar = d.uL[2 * ((j >> 1) * 2 + (i >> 1))]; ai = d.uL[2 * ((j >> 1) * 2 + (i >> 1)) + 1]; }
                if (d.uR) { br = d.uR[2 * ((j & 1) * 2 + (i & 1))]; bi = d.uR[2 * ((j & 1) * 2 + (i & 1)) + 1]; }
                kr = ar * br - ai * bi; ki = ar * bi + ai * br;
            }
            re += gr * kr - gi * ki; im += gr * ki + gi * kr;
        }
        Gs[tid].x = (float)re; Gs[tid].y = (float)im;
    }
    const C* A = (const C*)d.siteA;
    const C* B = (const C*)d.siteB;
    float p1[2][2][2][2], p2[2][2][2][2], p3[2][2][2][2];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        (&p1[0][0][0][0])[i] = 0.f; (&p2[0][0][0][0])[i] = 0.f; (&p3[0][0][0][0])[i] = 0.f;
    }
    const int a_row = tid >> 2, a_k = (tid & 3) * 4;
    const int b_k = tid >> 4, b_seg = tid & 15;
    const int b_dd = b_seg >> 3, b_r = (b_seg & 7) * 4;
    const int m = 2 * chiL;
    for (int k0 = 0; k0 < chiM; k0 += TH_K) {
        {
            const int grow = 2 * l0 + a_row;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + a_k + e;
                C v; v.x = 0; v.y = 0;
                if (grow < m && k < chiM) v = A[(size_t)grow * chiM + k];
                As[a_k + e][a_row] = make_float3(v.x, v.y, v.x + v.y);
            }
            const int k = k0 + b_k;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = r0 + b_r + e;
                C v; v.x = 0; v.y = 0;
                if (k < chiM && r < chiR) v = B[((size_t)k * 2 + b_dd) * chiR + r];
                Bs[b_k][b_dd * TH_R + b_r + e] = make_float3(v.x, v.y, v.x + v.y);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TH_K; ++kk) {
            float3 a[2][2], b[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                a[i][0] = As[kk][2 * (tx + 16 * i)];
                a[i][1] = As[kk][2 * (tx + 16 * i) + 1];
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                b[j][0] = Bs[kk][ty + 16 * j];
                b[j][1] = Bs[kk][TH_R + ty + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            p1[i][j][c][e] = fmaf(a[i][c].x, b[j][e].x, p1[i][j][c][e]);
                            p2[i][j][c][e] = fmaf(a[i][c].y, b[j][e].y, p2[i][j][c][e]);
                            p3[i][j][c][e] = fmaf(a[i][c].z, b[j][e].z, p3[i][j][c][e]);
                        }
        }
        __syncthreads();
    }
    C* Wm = (C*)d.W;
    C* T0 = (C*)d.theta0;
    SqAcc<float> fsq;  // |theta|_F^2 of this thread's elements
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int l = l0 + tx + 16 * i;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + ty + 16 * j;
            if (l < chiL && r < chiR) {
                C acc[2][2];
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        acc[c][e].x = p1[i][j][c][e] - p2[i][j][c][e];
                        acc[c][e].y = p3[i][j][c][e] - p1[i][j][c][e] - p2[i][j][c][e];
                    }
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) {
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa) {
                        C t; t.x = 0; t.y = 0;
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int e = 0; e < 2; ++e) cfma(t, Gs[(2 * aa + bb) * 4 + 2 * c + e], acc[c][e]);
                        const size_t idx = (size_t)(bb * chiR + r) * m + 2 * l + aa;
                        Wm[idx] = t;
                        T0[idx] = t;
                        fsq.add(t.x);
                        fsq.add(t.y);
                    }
                }
            }
        }
    }
    double fro = fsq.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0 && fro != 0.0) atomicAdd(&d.out->frob2, fro);
}

cudaError_t launch_theta_3m(const GateDesc* d, int n_gates, int chiL_max, int chiR_max, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    dim3 grid((chiL_max + TH_L - 1) / TH_L, (chiR_max + TH_R - 1) / TH_R, n_gates);
    k_theta_3m<<<grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

template cudaError_t launch_theta<float>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_theta<double>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_right<float>(const GateDesc*, int, int, int, cudaStream_t);
template cudaError_t launch_right<double>(const GateDesc*, int, int, int, cudaStream_t);

}  // namespace tnsim
