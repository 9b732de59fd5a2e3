// common.cuh - complex helpers, grid geometry and launch bookkeeping shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lsm {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };

template <typename C> struct real_of;
template <> struct real_of<float2> { typedef float type; };
template <> struct real_of<double2> { typedef double type; };

template <typename C> __host__ __device__ __forceinline__ C mkc(typename real_of<C>::type re, typename real_of<C>::type im) {
    C r; r.x = re; r.y = im; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// FP32 complex add/sub as one packed instruction each (add/sub.rn.f32x2, sm_100 family): the same
// IEEE rounding per lane, half the issue slots of two scalar operations.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) {
    C r; r.x = a.x * s; r.y = a.y * s; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
// multiply by (s * i), s = +1 or -1
template <int S, typename C> __device__ __forceinline__ C cmul_si(C a) {
    C r;
    if (S > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
template <typename C> __device__ __forceinline__ C from_d2(double2 a);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }

// Sign flips by XOR of the IEEE sign bit (m = 0 or SIGN_BIT), on the integer pipe.
constexpr unsigned SIGN_BIT = 0x80000000u;
__device__ __forceinline__ float flip_sign(float v, unsigned m) { return __uint_as_float(__float_as_uint(v) ^ m); }
__device__ __forceinline__ double flip_sign(double v, unsigned m) {
    return __hiloint2double(__double2hiint(v) ^ (int)m, __double2loint(v));
}
__device__ __forceinline__ float2 flip_sign(float2 v, unsigned m) { return make_float2(flip_sign(v.x, m), flip_sign(v.y, m)); }
__device__ __forceinline__ double2 flip_sign(double2 v, unsigned m) {
    return make_double2(flip_sign(v.x, m), flip_sign(v.y, m));
}

// g0 qa + g1 qb + g2 qc (conj(g) for CONJ) as two chains of one multiply and five FMAs.
template <bool CONJ, typename C>
__device__ __forceinline__ C gdot3(C g0, C qa, C g1, C qb, C g2, C qc) {
    typedef typename real_of<C>::type R;
    const R s = CONJ ? (R)-1 : (R)1;
    const R re = g0.x * qa.x - (s * g0.y) * qa.y + g1.x * qb.x - (s * g1.y) * qb.y + g2.x * qc.x - (s * g2.y) * qc.y;
    const R im = g0.x * qa.y + (s * g0.y) * qa.x + g1.x * qb.y + (s * g1.y) * qb.x + g2.x * qc.y + (s * g2.y) * qc.x;
    return mkc<C>(re, im);
}

// Shared-memory load the compiler may not merge with other loads of the same address or move:
// re-reading a small table at every use costs less than holding it in registers.
__device__ __forceinline__ float2 lds_fresh(const float2* p) {
    float2 r;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(r.x), "=f"(r.y) : "r"(a));
    return r;
}

// Asynchronous global -> shared copies (sm_80+ cp.async): 8- or 16-byte elements.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem_dst, const C* gmem_src) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem_dst);
    if (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// wait until at most N of the most recently committed groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Grid geometry of one medium.  Model nodes n_a; padded periodic length L_a = 2 n_a;
// extended contrast-source nodes e_a = n_a + 2 (nodes -1 .. n_a).
struct Dims {
    int nx, ny, nz;
    int Lx, Ly, Lz;
    int ex, ey, ez;
    long long N;      // nx*ny*nz
    double h;
};

// Shared-memory FFT plan of one length.  radix[] are the Stockham stages in order.
struct FftPlan {
    int L;
    int nst;
    int radix[12];
};

}  // namespace lsm
