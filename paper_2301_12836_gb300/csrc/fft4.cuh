// fft4.cuh - compile-time two-step ("four-step") FFT of lines held in shared memory.
//
// A line of length L = A * B is transformed as
//   Y[t][k1] = W_L^(t k1) * sum_a x[t + B a] W_A^(a k1)      (B DFTs of length A, then twiddles)
//   X[k1 + A k2] = sum_t Y[t][k1] W_B^(t k2)                  (A DFTs of length B)
// with every short DFT held in registers.  Each of the two steps reads its inputs from shared
// memory into registers, synchronises, and writes its outputs back in place, so one buffer of
// L * LD elements suffices.  A tile of NL lines is transformed by exactly NL * min(A, B)
// threads: thread tid works on line tid % NL.  Line l, element e sits at s[e * LD + l].
#pragma once
#include "fft.cuh"

namespace lsm {

template <int S, typename C>
__device__ __forceinline__ C cmul_const(C a, double re, double im_s) {
    // multiply by (re + S * i * im_s)
    typedef typename real_of<C>::type T;
    const T cr = (T)re, ci = (T)(S * im_s);
    return mkc<C>(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
}

// 16-point DFT in registers, natural order in and out: n = 4 n1 + n2, k = k1 + 4 k2.
// HALF: inputs 8..15 are zero, i.e. n1 = 2, 3 vanish in every first-layer 4-point DFT.
template <int S, bool HALF = false, typename C> __device__ __forceinline__ void bfly16(C* v) {
    const double c1 = 0.92387953251128675613;  // cos(pi/8)
    const double s1 = 0.38268343236508977173;  // sin(pi/8)
    const double r2 = 0.70710678118654752440;  // 1/sqrt(2)
    C y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        if (HALF) bfly4_half<S>(a);
        else bfly4<S>(a);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2 * 4 + k1] = a[k1];
    }
    // twiddles W16^(n2 k1), W16^m = cos(2 pi m/16) + S i sin(2 pi m/16)
    y[5] = cmul_const<S>(y[5], c1, s1);      // m = 1
    y[6] = cmul_const<S>(y[6], r2, r2);      // m = 2
    y[7] = cmul_const<S>(y[7], s1, c1);      // m = 3
    y[9] = cmul_const<S>(y[9], r2, r2);      // m = 2
    y[10] = cmul_si<S>(y[10]);               // m = 4
    y[11] = cmul_const<S>(y[11], -r2, r2);   // m = 6
    y[13] = cmul_const<S>(y[13], s1, c1);    // m = 3
    y[14] = cmul_const<S>(y[14], -r2, r2);   // m = 6
    y[15] = cmul_const<S>(y[15], -c1, -s1);  // m = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C b[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
        bfly4<S>(b);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
}

// 16-point DFT whose inputs NZ..15 are zero, computing only its first NO outputs: the zero
// inputs drop out of the first-layer 4-point DFTs, the unneeded outputs out of the last-layer
// ones.  NZ = NO = 16 is bfly16 operation for operation.
template <int S, int NZ, int N2, typename C> __device__ __forceinline__ void b16_first(const C* v, C* y) {
    constexpr int nz = (NZ - N2 + 3) / 4 < 1 ? 0 : ((NZ - N2 + 3) / 4 > 4 ? 4 : (NZ - N2 + 3) / 4);
    C a[4];
    if constexpr (nz == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = czero<C>();
    } else {
#pragma unroll
        for (int k = 0; k < nz; ++k) a[k] = v[N2 + 4 * k];
        bfly4p<S, nz, 4>(a);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[N2 * 4 + k1] = a[k1];
}
template <int S, int NO, int K1, typename C> __device__ __forceinline__ void b16_last(const C* y, C* v) {
    constexpr int no = (NO - K1 + 3) / 4 < 1 ? 0 : ((NO - K1 + 3) / 4 > 4 ? 4 : (NO - K1 + 3) / 4);
    if constexpr (no > 0) {
        C b[4] = {y[K1], y[4 + K1], y[8 + K1], y[12 + K1]};
        bfly4p<S, 4, no>(b);
#pragma unroll
        for (int k2 = 0; k2 < no; ++k2) v[K1 + 4 * k2] = b[k2];
    }
}
template <int S, int NZ, int NO, typename C> __device__ __forceinline__ void bfly16p(C* v) {
    const double c1 = 0.92387953251128675613;  // cos(pi/8)
    const double s1 = 0.38268343236508977173;  // sin(pi/8)
    const double r2 = 0.70710678118654752440;  // 1/sqrt(2)
    C y[16];
    b16_first<S, NZ, 0>(v, y);
    b16_first<S, NZ, 1>(v, y);
    b16_first<S, NZ, 2>(v, y);
    b16_first<S, NZ, 3>(v, y);
    // twiddles W16^(n2 k1), as in bfly16
    y[5] = cmul_const<S>(y[5], c1, s1);
    y[6] = cmul_const<S>(y[6], r2, r2);
    y[7] = cmul_const<S>(y[7], s1, c1);
    y[9] = cmul_const<S>(y[9], r2, r2);
    y[10] = cmul_si<S>(y[10]);
    y[11] = cmul_const<S>(y[11], -r2, r2);
    y[13] = cmul_const<S>(y[13], s1, c1);
    y[14] = cmul_const<S>(y[14], -r2, r2);
    y[15] = cmul_const<S>(y[15], -c1, -s1);
    b16_last<S, NO, 0>(y, v);
    b16_last<S, NO, 1>(y, v);
    b16_last<S, NO, 2>(y, v);
    b16_last<S, NO, 3>(y, v);
}

// W32^k a, W32^k = cos(2 pi k/32) + S i sin(2 pi k/32), k < 16 a compile-time constant after
// unrolling
template <int S, typename C> __device__ __forceinline__ C tw32(C a, int k) {
    const double c1 = 0.98078528040323044913, s1 = 0.19509032201612826785;  // cos, sin(pi/16)
    const double c2 = 0.92387953251128675613, s2 = 0.38268343236508977173;  // cos, sin(pi/8)
    const double c3 = 0.83146961230254523708, s3 = 0.55557023301960222474;  // cos, sin(3 pi/16)
    const double r2 = 0.70710678118654752440;
    switch (k) {
        case 0: return a;
        case 1: return cmul_const<S>(a, c1, s1);
        case 2: return cmul_const<S>(a, c2, s2);
        case 3: return cmul_const<S>(a, c3, s3);
        case 4: return cmul_const<S>(a, r2, r2);
        case 5: return cmul_const<S>(a, s3, c3);
        case 6: return cmul_const<S>(a, s2, c2);
        case 7: return cmul_const<S>(a, s1, c1);
        case 8: return cmul_si<S>(a);
        case 9: return cmul_const<S>(a, -s1, c1);
        case 10: return cmul_const<S>(a, -s2, c2);
        case 11: return cmul_const<S>(a, -s3, c3);
        case 12: return cmul_const<S>(a, -r2, r2);
        case 13: return cmul_const<S>(a, -c3, s3);
        case 14: return cmul_const<S>(a, -c2, s2);
        default: return cmul_const<S>(a, -c1, s1);
    }
}

// 32-point DFT in registers, natural order in and out, inputs NZ..31 zero and only the first NO
// outputs wanted: radix 2 over the 16-point DFTs E of the even and O of the odd samples,
// X[k] = E[k] + W32^k O[k] and X[k + 16] = E[k] - W32^k O[k] (k < 16).  The even samples keep
// (NZ + 1) / 2 nonzero inputs, the odd ones NZ / 2, and both halves need outputs k < min(NO, 16).
template <int S, int NZ, int NO, typename C> __device__ __forceinline__ void bfly32p(C* v) {
    constexpr int NZE = (NZ + 1) / 2, NZO = NZ / 2, NH = NO < 16 ? NO : 16;
    C e[16], o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        e[j] = v[2 * j];
        o[j] = v[2 * j + 1];
    }
    bfly16p<S, NZE, NH>(e);
    if constexpr (NZO >= 1) bfly16p<S, NZO, NH>(o);
#pragma unroll
    for (int k = 0; k < NH; ++k) {
        const C t = NZO >= 1 ? tw32<S>(o[k], k) : czero<C>();
        v[k] = cadd(e[k], t);
        if (k + 16 < NO) v[k + 16] = csub(e[k], t);
    }
}

// R-point DFT with inputs NZ..R-1 zero and only the first NO outputs needed.  Pruned forms exist
// for R = 32, 16 and 4 (and R = 8 with NZ <= 4, R = 2 with NZ = 1); otherwise the full DFT runs.
template <int R, int S, int NZ, int NO, typename C> __device__ __forceinline__ void dft_reg_p(C* v) {
    if constexpr (R == 32) {
        bfly32p<S, NZ, NO>(v);
    } else if constexpr (R == 16) {
        bfly16p<S, NZ, NO>(v);
    } else if constexpr (R == 4) {
        bfly4p<S, NZ, NO>(v);
    } else if constexpr (R == 8) {
        if constexpr (NZ <= 4) bfly8<S, true>(v);
        else bfly8<S>(v);
    } else {
        if constexpr (NZ == 1) v[1] = v[0];
        else bfly2<S>(v);
    }
}

// R-point DFT in registers; HALF: inputs R/2 .. R-1 are zero.
template <int R, int S, bool HALF = false, typename C> __device__ __forceinline__ void dft_reg(C* v) {
    if constexpr (R == 32) {
        bfly32p<S, HALF ? 16 : 32, 32>(v);
    } else if (R == 2) {
        if (HALF) v[1] = v[0];
        else bfly2<S>(v);
    } else if (R == 4) {
        if (HALF) bfly4_half<S>(v);
        else bfly4<S>(v);
    } else if (R == 8) {
        bfly8<S, HALF>(v);
    } else {
        bfly16<S, HALF>(v);
    }
}

template <int A, int B> struct FourStep {
    static constexpr int L = A * B;
    static constexpr int TPL = A < B ? A : B;   // threads per line
    static constexpr int I1 = B / TPL;          // step-1 DFTs per thread
    static constexpr int I2 = A / TPL;          // step-2 DFTs per thread
};

// In-place FFT (sign S) of NL lines; called by exactly NL * TPL threads, tid < NL * TPL.
// The caller synchronises before (input written) and gets the result after the final barrier.
// Zero padding and cropping are pruned at compile time: elements e >= NZ * B of a line are known
// to be zero (each step-1 DFT has at most NZ nonzero inputs), and only outputs k < NO * A are
// wanted (each step-2 DFT produces its first NO outputs; the others are left unwritten).
template <int A, int B, int S, int NZ = A, int NO = B, typename C>
__device__ __forceinline__ void fft4_smem(C* s, int NL, int LD, const C* __restrict__ tw, int tid) {
    typedef FourStep<A, B> F;
    const int l = tid % NL;
    const int q = tid / NL;
    C v[F::I1][A];
#pragma unroll
    for (int i = 0; i < F::I1; ++i) {
        const int t = q + F::TPL * i;
#pragma unroll
        for (int a = 0; a < A; ++a) v[i][a] = a < NZ ? s[(t + B * a) * LD + l] : czero<C>();
        dft_reg_p<A, S, NZ, A>(v[i]);
        if (t) {
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) {
                C w = __ldg(&tw[t * k1]);
                if (S > 0) w.y = -w.y;
                v[i][k1] = cmul(v[i][k1], w);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < F::I1; ++i) {
        const int t = q + F::TPL * i;
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) s[(t * A + k1) * LD + l] = v[i][k1];
    }
    __syncthreads();
    C w2[F::I2][B];
#pragma unroll
    for (int i = 0; i < F::I2; ++i) {
        const int k1 = q + F::TPL * i;
#pragma unroll
        for (int t = 0; t < B; ++t) w2[i][t] = s[(t * A + k1) * LD + l];
        dft_reg_p<B, S, B, NO>(w2[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < F::I2; ++i) {
        const int k1 = q + F::TPL * i;
#pragma unroll
        for (int k2 = 0; k2 < NO; ++k2) s[(k1 + A * k2) * LD + l] = w2[i][k2];
    }
    __syncthreads();
}

}  // namespace lsm

namespace lsm {

// Row stride (in elements) of the step-1 intermediate Y[t][k1] of fft4_io.  Threads of a warp
// write Y for consecutive t (groups of NL lanes) and read it back for consecutive k1; the skew
// PAD makes each group start on the banks where the previous one ended, so both accesses cost
// the minimum number of shared-memory wavefronts.  E = elements per 128-byte bank row.
template <int A, int E>
__host__ __device__ constexpr int fft4_pad(int NL) {
    return ((NL - A * NL) % E + E) % E;
}
template <int A, typename C>
__host__ __device__ constexpr int fft4_ystride(int NL) {
    return A * NL + fft4_pad<A, (int)(128 / sizeof(C))>(NL);
}

// Four-step FFT with caller-supplied input and output.  ld(l, e) returns element e of line l
// (IN_SMEM: it reads the buffer s itself, so a barrier separates those reads from the first
// write into s); st(l, k, v) receives output k of line l (OUT_SMEM: it writes s, so a barrier
// separates the last reads of s from those writes).  Called by exactly NL * TPL threads.  The
// intermediate occupies B * fft4_ystride<A, C>(NL) elements of s.  As in fft4_smem, inputs
// e >= NZ * B are known to be zero (ld is not called for them) and only outputs k < NO * A are
// produced (st is not called for the others).
template <int A, int B, int S, bool IN_SMEM, bool OUT_SMEM, int NL, int NZ = A, int NO = B, typename C, class Ld,
          class St>
__device__ __forceinline__ void fft4_io(C* s, const C* __restrict__ tw, int tid, Ld ld, St st) {
    typedef FourStep<A, B> F;
    const int l = tid % NL;
    const int q = tid / NL;
    constexpr int YS = fft4_ystride<A, C>(NL);
    C v[F::I1][A];
#pragma unroll
    for (int i = 0; i < F::I1; ++i) {
        const int t = q + F::TPL * i;
#pragma unroll
        for (int a = 0; a < A; ++a) v[i][a] = a < NZ ? ld(l, t + B * a) : czero<C>();
    }
#pragma unroll
    for (int i = 0; i < F::I1; ++i) {
        const int t = q + F::TPL * i;
        dft_reg_p<A, S, NZ, A>(v[i]);
        if (t) {
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) {
                C w = __ldg(&tw[t * k1]);
                if (S > 0) w.y = -w.y;
                v[i][k1] = cmul(v[i][k1], w);
            }
        }
    }
    if (IN_SMEM) __syncthreads();
#pragma unroll
    for (int i = 0; i < F::I1; ++i) {
        const int t = q + F::TPL * i;
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) s[t * YS + k1 * NL + l] = v[i][k1];
    }
    __syncthreads();
    C w2[F::I2][B];
#pragma unroll
    for (int i = 0; i < F::I2; ++i) {
        const int k1 = q + F::TPL * i;
#pragma unroll
        for (int t = 0; t < B; ++t) w2[i][t] = s[t * YS + k1 * NL + l];
        dft_reg_p<B, S, B, NO>(w2[i]);
    }
    if (OUT_SMEM) __syncthreads();
#pragma unroll
    for (int i = 0; i < F::I2; ++i) {
        const int k1 = q + F::TPL * i;
#pragma unroll
        for (int k2 = 0; k2 < NO; ++k2) st(l, k1 + A * k2, w2[i][k2]);
    }
    if (OUT_SMEM) __syncthreads();
}

}  // namespace lsm
