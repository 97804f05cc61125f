// Read-out of an MPS: amplitudes <x|psi> and transfer-matrix steps for <psi|P|psi>.
//
//  k_amplitudes : <x|psi> = A_0[x_0] A_1[x_1] ... A_{n-1}[x_{n-1}] (Eq. 2 with every
//                 physical leg fixed): one CTA per bitstring carries the row vector
//                 v (<= chi entries, shared memory) across the chain; each step is a
//                 vector-matrix product whose matrix rows are read coalesced.
//  k_tl1/k_tl2  : left transfer with a one-qubit operator O on site q,
//                 E'[a,b] = sum_{x,y,p,p'} conj(A[x,p,a]) O[p,p'] E[x,y] A[y,p',b].
//  k_tr1/k_tr2  : right transfer, R'[x,y] = sum conj(A[x,p,a]) O[p,p'] A[y,p',b] R[a,b];
//                 right environments are stored transposed (Rt[b][a]).
#include "tnsim_internal.h"

namespace tnsim {

template <typename C> __device__ __forceinline__ void cfma_(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ void cfmaconj_(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_amplitudes(void* const* __restrict__ sites,
                                                    const int* __restrict__ chi, int n,
                                                    const uint8_t* __restrict__ bits,
                                                    double* __restrict__ amps, int chi_cap) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* v0 = reinterpret_cast<C*>(smem_raw);
    C* v1 = v0 + chi_cap;
    const int64_t s = blockIdx.x;
    if (threadIdx.x == 0) { v0[0].x = 1; v0[0].y = 0; }
    __syncthreads();
    for (int q = 0; q < n; ++q) {
        const int x = bits[s * n + q] ? 1 : 0;
        const int cl = chi[q], cr = chi[q + 1];
        const C* A = (const C*)sites[q];
        for (int r = threadIdx.x; r < cr; r += blockDim.x) {
            C acc; acc.x = 0; acc.y = 0;
            for (int l = 0; l < cl; ++l) cfma_(acc, v0[l], A[(size_t)(2 * l + x) * cr + r]);
            v1[r] = acc;
        }
        __syncthreads();
        C* t = v0; v0 = v1; v1 = t;
    }
    if (threadIdx.x == 0) {
        amps[2 * s] = (double)v0[0].x;
        amps[2 * s + 1] = (double)v0[0].y;
    }
}

template <typename T>
cudaError_t launch_amplitudes(void* const* sites, const int* chi, int n_qubits, int chi_cap,
                              const uint8_t* bits, int64_t n_str, double* amps, cudaStream_t s) {
    using C = typename CT<T>::type;
    if (n_str <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)chi_cap * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_amplitudes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_amplitudes<T><<<(unsigned)n_str, 256, smem, s>>>(sites, chi, n_qubits, bits, amps, chi_cap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// left transfer: tmp[x, col] = sum_y E[x, y] A[y, col]  (col = p' * cr + b)
template <typename T>
__global__ void k_tl1(const typename CT<T>::type* __restrict__ A, const int* __restrict__ chi, int q,
                      const typename CT<T>::type* __restrict__ E, typename CT<T>::type* __restrict__ tmp) {
    using C = typename CT<T>::type;
    const int cl = chi[q], cr = chi[q + 1];
    const int ncol = 2 * cr;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)cl * ncol) return;
    const int x = (int)(t / ncol), col = (int)(t - (int64_t)x * ncol);
    C acc; acc.x = 0; acc.y = 0;
    for (int y = 0; y < cl; ++y) cfma_(acc, E[(size_t)x * cl + y], A[(size_t)y * ncol + col]);
    tmp[t] = acc;
}
// E'[a, b] = sum_{x,p} conj(A[x,p,a]) sum_{p'} O[p,p'] tmp[x, p', b]
template <typename T>
__global__ void k_tl2(const typename CT<T>::type* __restrict__ A, const int* __restrict__ chi, int q,
                      const double* __restrict__ op, const typename CT<T>::type* __restrict__ tmp,
                      typename CT<T>::type* __restrict__ Eo) {
    using C = typename CT<T>::type;
    const int cl = chi[q], cr = chi[q + 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)cr * cr) return;
    const int a = (int)(t / cr), b = (int)(t - (int64_t)a * cr);
    C o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { o[i].x = (T)op[2 * i]; o[i].y = (T)op[2 * i + 1]; }
    C acc; acc.x = 0; acc.y = 0;
    for (int x = 0; x < cl; ++x) {
        const C t0 = tmp[(size_t)x * 2 * cr + b], t1 = tmp[(size_t)x * 2 * cr + cr + b];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            C w; w.x = 0; w.y = 0;
            cfma_(w, o[2 * p], t0);
            cfma_(w, o[2 * p + 1], t1);
            cfmaconj_(acc, A[(size_t)(2 * x + p) * cr + a], w);
        }
    }
    Eo[t] = acc;
}

// right transfer with Rt[b][a] = R[a][b] (a: bra, b: ket on bond q+1):
// tmp[y, p', a] = sum_b A[y, p', b] Rt[b, a]
template <typename T>
__global__ void k_tr1(const typename CT<T>::type* __restrict__ A, const int* __restrict__ chi, int q,
                      const typename CT<T>::type* __restrict__ Rt, typename CT<T>::type* __restrict__ tmp) {
    using C = typename CT<T>::type;
    const int cl = chi[q], cr = chi[q + 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)cl * 2 * cr) return;
    const int row = (int)(t / cr), a = (int)(t - (int64_t)row * cr);   // row = y*2 + p'
    C acc; acc.x = 0; acc.y = 0;
    for (int b = 0; b < cr; ++b) cfma_(acc, A[(size_t)row * cr + b], Rt[(size_t)b * cr + a]);
    tmp[t] = acc;
}
// Rt'[y, x] = R'[x, y] = sum_{p,a} conj(A[x,p,a]) sum_{p'} O[p,p'] tmp[y,p',a]
template <typename T>
__global__ void k_tr2(const typename CT<T>::type* __restrict__ A, const int* __restrict__ chi, int q,
                      const double* __restrict__ op, const typename CT<T>::type* __restrict__ tmp,
                      typename CT<T>::type* __restrict__ Rto) {
    using C = typename CT<T>::type;
    const int cl = chi[q], cr = chi[q + 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)cl * cl) return;
    const int y = (int)(t / cl), x = (int)(t - (int64_t)y * cl);
    C o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { o[i].x = (T)op[2 * i]; o[i].y = (T)op[2 * i + 1]; }
    C acc; acc.x = 0; acc.y = 0;
    for (int a = 0; a < cr; ++a) {
        const C t0 = tmp[(size_t)(2 * y) * cr + a], t1 = tmp[(size_t)(2 * y + 1) * cr + a];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            C w; w.x = 0; w.y = 0;
            cfma_(w, o[2 * p], t0);
            cfma_(w, o[2 * p + 1], t1);
            cfmaconj_(acc, A[(size_t)(2 * x + p) * cr + a], w);
        }
    }
    Rto[t] = acc;
}

template <typename T>
cudaError_t launch_transfer(const void* site, const int* chi, int q, const double* op,
                            const void* e_in, void* tmp, void* e_out, int chi_cap,
                            int from_left, cudaStream_t s) {
    using C = typename CT<T>::type;
    const int64_t n1 = (int64_t)chi_cap * 2 * chi_cap;
    const int64_t n2 = (int64_t)chi_cap * chi_cap;
    const unsigned g1 = (unsigned)((n1 + 255) / 256), g2 = (unsigned)((n2 + 255) / 256);
    if (from_left) {
        k_tl1<T><<<g1, 256, 0, s>>>((const C*)site, chi, q, (const C*)e_in, (C*)tmp);
        k_tl2<T><<<g2, 256, 0, s>>>((const C*)site, chi, q, op, (const C*)tmp, (C*)e_out);
    } else {
        k_tr1<T><<<g1, 256, 0, s>>>((const C*)site, chi, q, (const C*)e_in, (C*)tmp);
        k_tr2<T><<<g2, 256, 0, s>>>((const C*)site, chi, q, op, (const C*)tmp, (C*)e_out);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_rt(const void* site, const int* chi, int q, const void* rt, void* tmp, int chi_cap,
                            cudaStream_t s) {
    using C = typename CT<T>::type;
    const int64_t n1 = (int64_t)chi_cap * 2 * chi_cap;
    k_tr1<T><<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>((const C*)site, chi, q, (const C*)rt, (C*)tmp);
    return cudaGetLastError();
}
template cudaError_t launch_apply_rt<float>(const void*, const int*, int, const void*, void*, int, cudaStream_t);
template cudaError_t launch_apply_rt<double>(const void*, const int*, int, const void*, void*, int, cudaStream_t);

// <L | R>-style closure: out = sum_{x,y} E[x,y] Rt[y,x] over one bond, E and Rt both chi x chi
template <typename T>
__global__ void k_close(const typename CT<T>::type* __restrict__ E, const typename CT<T>::type* __restrict__ Rt,
                        const int* __restrict__ chi, int bond, double* __restrict__ out) {
    using C = typename CT<T>::type;
    const int c = chi[bond];
    double re = 0.0, im = 0.0;
    for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
        const int x = t / c, y = t - x * c;
        const C e = E[(size_t)x * c + y], r = Rt[(size_t)y * c + x];
        re += (double)e.x * r.x - (double)e.y * r.y;
        im += (double)e.x * r.y + (double)e.y * r.x;
    }
    __shared__ double sr[256], si[256];
    sr[threadIdx.x] = re; si[threadIdx.x] = im;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { sr[threadIdx.x] += sr[threadIdx.x + o]; si[threadIdx.x] += si[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sr[0]; out[1] = si[0]; }
}

template <typename T>
cudaError_t launch_close(const void* E, const void* Rt, const int* chi, int bond, double* out,
                         cudaStream_t s) {
    using C = typename CT<T>::type;
    k_close<T><<<1, 256, 0, s>>>((const C*)E, (const C*)Rt, chi, bond, out);
    return cudaGetLastError();
}

template cudaError_t launch_amplitudes<float>(void* const*, const int*, int, int, const uint8_t*, int64_t, double*, cudaStream_t);
template cudaError_t launch_amplitudes<double>(void* const*, const int*, int, int, const uint8_t*, int64_t, double*, cudaStream_t);
template cudaError_t launch_transfer<float>(const void*, const int*, int, const double*, const void*, void*, void*, int, int, cudaStream_t);
template cudaError_t launch_transfer<double>(const void*, const int*, int, const double*, const void*, void*, void*, int, int, cudaStream_t);
template cudaError_t launch_close<float>(const void*, const void*, const int*, int, double*, cudaStream_t);
template cudaError_t launch_close<double>(const void*, const void*, const int*, int, double*, cudaStream_t);

}  // namespace tnsim
