// reduce.cuh - deterministic two-stage reductions with FP64-accurate inner products and the
// alpha / omega steps of BiCGSTAB, for the vector kernels and the kernel that finishes the inner
// products summed in the operator epilogue (solver.cu).  Internal.
#pragma once
#include "solver.cuh"

namespace lsm {

// Sum v over the block into thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[wid * K + k] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = lane < nw ? sh[lane * K + k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            v[k] = a;
        }
    }
}

// Reduce v over the grid's x dimension for system sys.  Returns true in thread 0 of the last
// CTA, with tot holding the system's sums.
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], Partials pt, int sys, unsigned int* counter, double (&tot)[K]) {
    __shared__ double sh[32 * K];
    __shared__ int last;
    block_sum<K>(v, sh);
    if (threadIdx.x == 0) {
        double* dst = pt.buf + ((long long)sys * pt.nblk + blockIdx.x) * 4;
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = v[k];
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double* src = pt.buf + ((long long)sys * pt.nblk + b) * 4;
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] += __ldcg(&src[k]);
    }
    block_sum<K>(a, sh);
    if (threadIdx.x == 0) {
        *counter = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = a[k];
        return true;
    }
    return false;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Running inner-product sums of one thread, K of them.
// FP64 vectors: FP64 sums of FP64 products.
// FP32 vectors: each product of two FP32 numbers is split exactly into p = fl(a b) and
// e = fma(a, b, -p) (p + e = a b); p enters a compensated FP32 pair (hi, lo) through TwoSum, whose
// rounding error joins e in lo, and after every FLUSH elements (strided4_sum calls flush() at
// fixed points of its loop) the pair is added to an FP64 total.
// With at most 2 FLUSH products per sum between flushes, the partial pair is within about
// (4 FLUSH)^2 / 2 * 2^-48 (< 1e-11) of the exact sum, relative to the sum of |products|; the
// totals and the cross-thread reduction are FP64.  This keeps the reductions memory-bound
// instead of bound by the FP64 pipe (one 64th of the FP32 rate on this part).
template <typename C, int K> struct Sums;

template <int K> struct Sums<double2, K> {
    double d[K];
    __device__ __forceinline__ Sums() {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = 0.0;
    }
    static constexpr int FLUSH = 16;   // loop structure shared with the FP32 sums; nothing to flush
    __device__ __forceinline__ void prod(int k, double a, double b) { d[k] = fma(a, b, d[k]); }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ void finish(double (&out)[K]) {
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = d[k];
    }
};

// Knuth's TwoSum: s = fl(a + b) and a + b = s + e exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return s;
}

template <int K> struct Sums<float2, K> {
    static constexpr int FLUSH = 16;
    float hi[K], lo[K];
    double d[K];
    __device__ __forceinline__ Sums() {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            hi[k] = lo[k] = 0.f;
            d[k] = 0.0;
        }
    }
    __device__ __forceinline__ void prod(int k, float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float err;
        hi[k] = two_sum(hi[k], p, err);
        lo[k] = __fadd_rn(lo[k], __fadd_rn(err, e));
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            d[k] += (double)hi[k] + (double)lo[k];
            hi[k] = lo[k] = 0.f;
        }
    }
    __device__ __forceinline__ void finish(double (&out)[K]) {
        flush();
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = d[k];
    }
};

// sums k (re) and k + 1 (im) += conj(a) b
template <typename C, int K>
__device__ __forceinline__ void acc_dot(Sums<C, K>& S, int k, C a, C b) {
    S.prod(k, a.x, b.x);
    S.prod(k, a.y, b.y);
    S.prod(k + 1, a.x, b.y);
    S.prod(k + 1, -a.y, b.x);
}
// sum k += |a|^2
template <typename C, int K>
__device__ __forceinline__ void acc_nrm(Sums<C, K>& S, int k, C a) {
    S.prod(k, a.x, a.x);
    S.prod(k, a.y, a.y);
}

// alpha = rho / <r^, v> (Van der Vorst's BiCGSTAB, Sec. 3.2); a vanishing or non-finite ratio is a
// breakdown: the system stops with status -4.  tot = (Re, Im) of <r^, v>.
__device__ __forceinline__ void bcg_alpha_final(BcgState& S, const double* tot, int* n_active) {
    S.rv = make_double2(tot[0], tot[1]);
    const double2 a = cdiv(S.rho, S.rv);
    if ((tot[0] == 0.0 && tot[1] == 0.0) || !finite2(a)) {
        S.status = -4;
        S.active = S.run_v = S.run_t = 0;
        atomicSub(n_active, 1);
    } else {
        S.alpha = a;
    }
}

// omega = <t, s> / <t, t>; a zero <t, t> leaves omega = 0, caught as a breakdown by k_bcg_xr.
// tot = (Re, Im) of <t, s>, then <t, t>.
__device__ __forceinline__ void bcg_omega_final(BcgState& S, const double* tot) {
    S.ts = make_double2(tot[0], tot[1]);
    S.tt = tot[2];
    S.omega = tot[2] > 0.0 ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
}

}  // namespace lsm
