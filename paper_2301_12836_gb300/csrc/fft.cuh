// fft.cuh - batched Stockham FFT of lines held in shared memory.
//
// The convolution of Eq. 21 runs as three axis passes per direction.  Each
// pass stages a tile of lines in shared memory, transforms them there with
// the self-sorting Stockham formulation (Govindaraju et al., SC'08) in
// mixed radix 8/4/2/3/5, and writes them back.  Line l, element e of a
// tile lives at s[e * LD + l]: threads with consecutive indices work on
// consecutive lines, so every stage reads and writes shared memory without
// bank conflicts when LD is the tile width, and global rows of the tile
// (consecutive lines along x) are coalesced.
//
// Stage with radix R after Ns = product of the earlier radices: butterfly j
// (0 <= j < L/R) reads elements j + r L/R, multiplies element r by
// W^(r (j mod Ns) L/(Ns R)) with W = exp(dir 2 pi i / L), takes the R-point DFT
// and writes element (j div Ns) Ns R + (j mod Ns) + r Ns of the other buffer.
// Forward is dir = -1 (numpy's convention); inverse is dir = +1 and unnormalised.
#pragma once
#include "dfloat.cuh"

namespace lsm {

// R-point DFTs, sign S = dir.
template <int S, typename C> __device__ __forceinline__ void bfly2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}

template <int S, typename C> __device__ __forceinline__ void bfly4(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmul_si<S>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
}

// 4-point DFT whose inputs NZ..3 are zero (NZ = 1..4), computing only its first NO outputs
// (NO = 1..4); NZ = NO = 4 is bfly4 operation for operation.
template <int S, int NZ, int NO, typename C> __device__ __forceinline__ void bfly4p(C* v) {
    static_assert(NZ >= 1 && NZ <= 4 && NO >= 1 && NO <= 4, "bfly4p");
    if constexpr (NZ == 1) {
#pragma unroll
        for (int k = 1; k < NO; ++k) v[k] = v[0];
        return;
    } else {
        C t0, t1, t2, t3;
        if constexpr (NZ >= 3) {
            t0 = cadd(v[0], v[2]);
            t1 = csub(v[0], v[2]);
        } else {
            t0 = v[0];
            t1 = v[0];
        }
        if constexpr (NZ == 4) {
            t2 = cadd(v[1], v[3]);
            t3 = cmul_si<S>(csub(v[1], v[3]));
        } else {
            t2 = v[1];
            t3 = cmul_si<S>(v[1]);
        }
        v[0] = cadd(t0, t2);
        if constexpr (NO >= 2) v[1] = cadd(t1, t3);
        if constexpr (NO >= 3) v[2] = csub(t0, t2);
        if constexpr (NO >= 4) v[3] = csub(t1, t3);
    }
}

// 4-point DFT of (v0, v1, 0, 0): the first radix-2 layer has nothing to add.
template <int S, typename C> __device__ __forceinline__ void bfly4_half(C* v) {
    const C a = v[0], b = v[1], bi = cmul_si<S>(v[1]);
    v[0] = cadd(a, b); v[2] = csub(a, b);
    v[1] = cadd(a, bi); v[3] = csub(a, bi);
}

// HALF: inputs 4..7 are zero (zero-padded lines), so each 4-point half-DFT has two zero inputs.
template <int S, bool HALF = false, typename C> __device__ __forceinline__ void bfly8(C* v) {
    typedef typename real_of<C>::type T;
    const T r2 = (T)0.70710678118654752440;  // 1/sqrt(2)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    if (HALF) {
        bfly4_half<S>(e);
        bfly4_half<S>(o);
    } else {
        bfly4<S>(e);
        bfly4<S>(o);
    }
    // twiddles w^s, w = exp(S 2 pi i / 8)
    C o1 = mkc<C>((o[1].x - (T)S * o[1].y) * r2, (o[1].y + (T)S * o[1].x) * r2);     // * (1 + S i)/sqrt2
    C o2 = cmul_si<S>(o[2]);                                                          // * S i
    C o3 = mkc<C>((-o[3].x - (T)S * o[3].y) * r2, (-o[3].y + (T)S * o[3].x) * r2);   // * (-1 + S i)/sqrt2
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}

template <int S, typename C> __device__ __forceinline__ void bfly3(C* v) {
    typedef typename real_of<C>::type T;
    const T s3 = (T)0.86602540378443864676;  // sqrt(3)/2
    C t = cadd(v[1], v[2]);
    C d = cscale(cmul_si<S>(csub(v[1], v[2])), s3);
    C m = csub(v[0], cscale(t, (T)0.5));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, d);
    v[2] = csub(m, d);
}

template <int S, typename C> __device__ __forceinline__ void bfly5(C* v) {
    typedef typename real_of<C>::type T;
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi/5) = (sqrt5 - 1)/4
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi/5) = -(sqrt5 + 1)/4
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi/5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi/5)
    C a14 = cadd(v[1], v[4]), b14 = csub(v[1], v[4]);
    C a23 = cadd(v[2], v[3]), b23 = csub(v[2], v[3]);
    C m1 = cadd(v[0], cadd(cscale(a14, c1), cscale(a23, c2)));
    C m2 = cadd(v[0], cadd(cscale(a14, c2), cscale(a23, c1)));
    C n1 = cmul_si<S>(cadd(cscale(b14, s1), cscale(b23, s2)));
    C n2 = cmul_si<S>(csub(cscale(b14, s2), cscale(b23, s1)));
    v[0] = cadd(v[0], cadd(a14, a23));
    v[1] = cadd(m1, n1); v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2); v[3] = csub(m2, n2);
}

template <int S, int R, typename C>
__device__ __forceinline__ void fft_stage_r(const C* __restrict__ src, C* __restrict__ dst, int L, int Ns,
                                            int NL, int LD, const C* __restrict__ tw, int tid, int nth) {
    const int nb = L / R;
    const int total = nb * NL;
    const int tstep = L / (Ns * R);
    for (int it = tid; it < total; it += nth) {
        const int l = it % NL;
        const int j = it / NL;
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * LD + l];
        if (k) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = __ldg(&tw[r * k * tstep]);
                if (S > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 2) bfly2<S>(v);
        else if (R == 3) bfly3<S>(v);
        else if (R == 4) bfly4<S>(v);
        else if (R == 5) bfly5<S>(v);
        else bfly8<S>(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * LD + l] = v[r];
    }
}

// Transform NL lines of length p.L held in buffer a (layout s[e*LD + l]); b is scratch of the
// same size.  Returns the buffer holding the result.  The caller synchronises the block before
// the call; the result is visible to all threads on return.  tw = exp(-2 pi i k / L), k < L.
template <int S, typename C>
__device__ C* fft_smem(C* a, C* b, const FftPlan& p, int NL, int LD, const C* __restrict__ tw, int tid, int nth) {
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        switch (R) {
            case 8: fft_stage_r<S, 8>(a, b, p.L, Ns, NL, LD, tw, tid, nth); break;
            case 4: fft_stage_r<S, 4>(a, b, p.L, Ns, NL, LD, tw, tid, nth); break;
            case 2: fft_stage_r<S, 2>(a, b, p.L, Ns, NL, LD, tw, tid, nth); break;
            case 3: fft_stage_r<S, 3>(a, b, p.L, Ns, NL, LD, tw, tid, nth); break;
            default: fft_stage_r<S, 5>(a, b, p.L, Ns, NL, LD, tw, tid, nth); break;
        }
        __syncthreads();
        C* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace lsm
