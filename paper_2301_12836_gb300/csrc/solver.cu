// solver.cu - BiCGSTAB vector updates, FP64 inner products and the mixed-precision refinement
// kernels (Sec. 3.2, Eq. 22).
//
// Every reduction is two-stage and deterministic: each CTA reduces its slice with warp shuffles
// and writes one partial; the last CTA to finish (atomic ticket after a memory fence) sums the
// partials in block order and updates the system's scalars on the device.  Kernels of systems
// that stopped return at once, so a batch keeps launching one grid per step whatever its mix of
// converged and running systems.
#include "reduce.cuh"

namespace lsm {

static constexpr int VTH = 256;

int vec_blocks(long long n) {
    long long b = (n + VTH * 4 - 1) / (VTH * 4);
    if (b > 2 * 152) b = 2 * 152;
    if (b < 1) b = 1;
    return (int)b;
}

// Grid-stride loop over [0, n) in the order i0, i0 + S, i0 + 2 S, ... (S = threads of the grid's
// x dimension), four indices at a time: ld(i) reads element i's operands, use(i, v) consumes them
// in index order.  The four reads issue before the first use, so every thread keeps four
// independent loads in flight (one at a time left these streams latency-bound); each thread still
// visits its elements in the same order, so every sum is bitwise the same.
template <class Ld, class Use>
__device__ __forceinline__ void strided4(long long n, Ld ld, Use use) {
    const long long S = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * S < n; i += 4 * S) {
        const auto v0 = ld(i);
        const auto v1 = ld(i + S);
        const auto v2 = ld(i + 2 * S);
        const auto v3 = ld(i + 3 * S);
        use(i, v0);
        use(i + S, v1);
        use(i + 2 * S, v2);
        use(i + 3 * S, v3);
    }
    for (; i < n; i += S) use(i, ld(i));
}
// strided4 for the kernels that also sum: the elements go in the same order, and acc.flush()
// (compensated FP32 pairs into FP64 totals) runs after every Acc::FLUSH elements of the main loop
// as a fixed part of the loop.  (A counter test per element was if-converted by the compiler,
// which then issued the FP64 flush for every element and bound these streams by the FP64 pipe.)
template <class Acc, class Ld, class Use>
__device__ __forceinline__ void strided4_sum(long long n, Acc& acc, Ld ld, Use use) {
    constexpr int CH = Acc::FLUSH / 4;
    const long long S = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (4LL * CH - 1) * S < n;) {
#pragma unroll 1
        for (int c = 0; c < CH; ++c, i += 4 * S) {
            const auto v0 = ld(i);
            const auto v1 = ld(i + S);
            const auto v2 = ld(i + 2 * S);
            const auto v3 = ld(i + 3 * S);
            use(i, v0);
            use(i + S, v1);
            use(i + 2 * S, v2);
            use(i + 3 * S, v3);
        }
        acc.flush();
    }
    // fewer than FLUSH elements remain: no flush before the caller's finish()
    for (; i + 3 * S < n; i += 4 * S) {
        const auto v0 = ld(i);
        const auto v1 = ld(i + S);
        const auto v2 = ld(i + 2 * S);
        const auto v3 = ld(i + 3 * S);
        use(i, v0);
        use(i + S, v1);
        use(i + 2 * S, v2);
        use(i + 3 * S, v3);
    }
    for (; i < n; i += S) use(i, ld(i));
}
template <typename C> struct Two { C a, b; };
template <typename C> struct Three { C a, b, c; };

template <typename T>
__global__ void __launch_bounds__(VTH) k_bcg_init(const BcgVecs<T>* __restrict__ vecs, BcgState* __restrict__ st,
                                                  Partials pt, long long n, int x_zero, const MixState* __restrict__ skip,
                                                  int* n_active) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    if (skip && skip[sys].done) return;
    const BcgVecs<T> V = vecs[sys];
    Sums<C, 2> acc;
    strided4_sum(n, acc, [&](long long i) { return Two<C>{V.b[i], x_zero ? czero<C>() : V.v[i]}; },
                 [&](long long i, const Two<C>& w) {
                     const C r = x_zero ? w.a : csub(w.a, w.b);
                     V.r[i] = r;
                     V.rh[i] = r;
                     acc_nrm(acc, 0, w.a);
                     acc_nrm(acc, 1, r);
                 });
    double v[2], tot[2];
    acc.finish(v);
    if (grid_sum<2>(v, pt, sys, &st[sys].counter, tot)) {
        BcgState& S = st[sys];
        S.bnorm2 = tot[0];
        S.rnorm2 = tot[1];
        S.rho = make_double2(tot[1], 0.0);
        S.tol2 = S.tol2 * tot[0];
        S.iters = 0;
        S.half = 0;
        S.status = 0;
        S.active = (tot[0] > 0.0 && tot[1] > S.tol2) ? 1 : 0;
        S.run_v = S.run_t = S.active;
        if (S.active) atomicAdd(n_active, 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(VTH) k_bcg_p(const BcgVecs<T>* __restrict__ vecs, const BcgState* __restrict__ st, long long n) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    const BcgState& S = st[sys];
    if (!S.active) return;
    const BcgVecs<T> V = vecs[sys];
    if (S.iters == 0) {
        strided4(n, [&](long long i) { return V.r[i]; }, [&](long long i, const C& r) { V.p[i] = r; });
        return;
    }
    const C be = from_d2<C>(S.beta), om = from_d2<C>(S.omega);
    strided4(n, [&](long long i) { return Three<C>{V.p[i], V.v[i], V.r[i]}; },
             [&](long long i, const Three<C>& w) {
                 const C pv = csub(w.a, cmul(om, w.b));
                 V.p[i] = cadd(w.c, cmul(be, pv));
             });
}

template <typename T>
__global__ void __launch_bounds__(VTH) k_bcg_alpha(const BcgVecs<T>* __restrict__ vecs, BcgState* __restrict__ st,
                                                   Partials pt, long long n, int* n_active) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    if (!st[sys].run_v) return;
    const BcgVecs<T> V = vecs[sys];
    Sums<C, 2> acc;
    strided4_sum(n, acc, [&](long long i) { return Two<C>{V.rh[i], V.v[i]}; },
                 [&](long long, const Two<C>& w) {
                     acc_dot(acc, 0, w.a, w.b);
                 });
    double v[2], tot[2];
    acc.finish(v);
    if (grid_sum<2>(v, pt, sys, &st[sys].counter, tot)) bcg_alpha_final(st[sys], tot, n_active);
}

template <typename T>
__global__ void __launch_bounds__(VTH) k_bcg_s(const BcgVecs<T>* __restrict__ vecs, BcgState* __restrict__ st,
                                               Partials pt, long long n) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    if (!st[sys].active) return;
    const BcgVecs<T> V = vecs[sys];
    const C al = from_d2<C>(st[sys].alpha);
    Sums<C, 1> acc;
    strided4_sum(n, acc, [&](long long i) { return Two<C>{V.r[i], V.v[i]}; },
                 [&](long long i, const Two<C>& w) {
                     const C s = csub(w.a, cmul(al, w.b));
                     V.s[i] = s;
                     acc_nrm(acc, 0, s);
                 });
    double v[1], tot[1];
    acc.finish(v);
    if (grid_sum<1>(v, pt, sys, &st[sys].counter, tot)) {
        BcgState& S = st[sys];
        S.snorm2 = tot[0];
        if (tot[0] <= S.tol2) {
            S.half = 1;
            S.run_t = 0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(VTH) k_bcg_omega(const BcgVecs<T>* __restrict__ vecs, BcgState* __restrict__ st,
                                                   Partials pt, long long n) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    if (!st[sys].run_t) return;
    const BcgVecs<T> V = vecs[sys];
    Sums<C, 3> acc;
    strided4_sum(n, acc, [&](long long i) { return Two<C>{V.t[i], V.s[i]}; },
                 [&](long long, const Two<C>& w) {
                     acc_dot(acc, 0, w.a, w.b);
                     acc_nrm(acc, 2, w.a);
                 });
    double v[3], tot[3];
    acc.finish(v);
    if (grid_sum<3>(v, pt, sys, &st[sys].counter, tot)) bcg_omega_final(st[sys], tot);
}

// Sum the epilogue partials of each system's DotSink in FP64 (each thread a fixed stride of them,
// then the block tree: the same order every call) and finish alpha (DOT_RV) or omega (DOT_TS);
// one block per system, skipped like the apply that wrote them.
__global__ void __launch_bounds__(VTH) k_dot_finish(const DotSink* __restrict__ sinks) {
    const DotSink D = sinks[blockIdx.x];
    const bool rv = D.mode == DOT_RV;
    if (!(rv ? D.st->run_v : D.st->run_t)) return;
    __shared__ double sh[32 * 3];
    double a[3] = {0.0, 0.0, 0.0};
    const float4* __restrict__ src = reinterpret_cast<const float4*>(D.partials);
    for (int b = threadIdx.x; b < D.nparts; b += blockDim.x) {
        const float4 p = __ldcg(&src[b]);
        a[0] += p.x;
        a[1] += p.y;
        a[2] += p.z;
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0) {
        if (rv) bcg_alpha_final(*D.st, a, D.n_active);
        else bcg_omega_final(*D.st, a);
    }
}

template <typename T>
__global__ void __launch_bounds__(VTH, sizeof(T) == 4 ? 3 : 2) k_bcg_xr(const BcgVecs<T>* __restrict__ vecs, BcgState* __restrict__ st,
                                                Partials pt, long long n, int* n_active) {
    typedef typename cplx_of<T>::type C;
    const int sys = blockIdx.y;
    if (!st[sys].active) return;
    const BcgVecs<T> V = vecs[sys];
    const int half = st[sys].half;
    const C al = from_d2<C>(st[sys].alpha);
    const C om = from_d2<C>(st[sys].omega);
    Sums<C, 3> acc;
    if (half) {
        strided4(n, [&](long long i) { return Two<C>{V.x[i], V.p[i]}; },
                 [&](long long i, const Two<C>& w) { V.x[i] = cadd(w.a, cmul(al, w.b)); });
    } else {
        struct Five { C s, t, x, p, rh; };
        strided4_sum(n, acc, [&](long long i) { return Five{V.s[i], V.t[i], V.x[i], V.p[i], V.rh[i]}; },
                     [&](long long i, const Five& w) {
                         V.x[i] = cadd(w.x, cadd(cmul(al, w.p), cmul(om, w.s)));
                         const C r = csub(w.s, cmul(om, w.t));
                         V.r[i] = r;
                         acc_nrm(acc, 0, r);
                         acc_dot(acc, 1, w.rh, r);
                     });
    }
    double v[3], tot[3];
    acc.finish(v);
    if (grid_sum<3>(v, pt, sys, &st[sys].counter, tot)) {
        BcgState& S = st[sys];
        S.iters += 1;
        if (half) {
            S.rnorm2 = S.snorm2;
            S.active = 0;
            S.status = 0;
        } else {
            S.rnorm2 = tot[0];
            const double2 rho_new = make_double2(tot[1], tot[2]);
            if (tot[0] <= S.tol2) {
                S.active = 0;
                S.status = 0;
            } else if ((S.omega.x == 0.0 && S.omega.y == 0.0) || (rho_new.x == 0.0 && rho_new.y == 0.0) ||
                       !finite2(rho_new) || !isfinite(tot[0])) {
                S.active = 0;
                S.status = -4;
            } else if (S.iters >= S.maxit) {
                S.active = 0;
                S.status = -5;
            } else {
                S.beta = cmuld(cdiv(rho_new, S.rho), cdiv(S.alpha, S.omega));
                S.rho = rho_new;
            }
        }
        S.half = 0;
        S.run_v = S.run_t = S.active;
        if (!S.active) atomicSub(n_active, 1);
    }
}

// ---------------------------------------------------------------------------------------------
// mixed-precision refinement
// ---------------------------------------------------------------------------------------------
// r = b - A x and the norms of b and r.  PAIR (double-float residual apply, x entered scaled by
// 2^-pexp): b is split into pairs at the same scale by integer operations, r = b - A x is one
// double-float subtraction on the FP32 pipe and is stored as pairs (rpair), and the norms sum the
// squares of the high words in FP32 per thread (relative error ~1e-6, all a convergence test and a
// normalisation need), totals in FP64.  Otherwise (FP64 apply, or x = 0 so that r = b): FP64.
template <bool PAIR>
__global__ void __launch_bounds__(VTH) k_mix_res(const double2* const* __restrict__ b, const double2* const* __restrict__ ax,
                                                 double2* const* __restrict__ r64, MixState* __restrict__ ms, Partials pt,
                                                 long long n, int* n_active) {
    const int sys = blockIdx.y;
    if (ms[sys].done) return;
    const double2* B = b[sys];
    const double2* AX = ax[sys];
    double2* R = r64[sys];
    const int xz = ms[sys].xzero;
    const bool pair = PAIR && !xz;
    const int pexp = ms[sys].pexp;
    double v[2] = {0.0, 0.0};
    if (pair) {
        float sb = 0.f, sr = 0.f;
        struct BA { double2 b; float4 a; };
        strided4(n, [&](long long i) { return BA{B[i], reinterpret_cast<const float4*>(AX)[i]}; },
                 [&](long long i, const BA& w) {
                     const dfloat br = df_split(w.b.x, pexp), bi = df_split(w.b.y, pexp);
                     const dfloat rr = br - dfloat(w.a.x, w.a.y), ri = bi - dfloat(w.a.z, w.a.w);
                     reinterpret_cast<float4*>(R)[i] = make_float4(rr.hi, rr.lo, ri.hi, ri.lo);
                     sb = __fmaf_rn(br.hi, br.hi, __fmaf_rn(bi.hi, bi.hi, sb));
                     sr = __fmaf_rn(rr.hi, rr.hi, __fmaf_rn(ri.hi, ri.hi, sr));
                 });
        v[0] = (double)sb;
        v[1] = (double)sr;
    } else {
        strided4(n, [&](long long i) { return Two<double2>{B[i], xz ? make_double2(0.0, 0.0) : AX[i]}; },
                 [&](long long i, const Two<double2>& w) {
                     const double2 r = make_double2(w.a.x - w.b.x, w.a.y - w.b.y);
                     R[i] = r;
                     v[0] += w.a.x * w.a.x + w.a.y * w.a.y;
                     v[1] += r.x * r.x + r.y * r.y;
                 });
    }
    double tot[2];
    if (grid_sum<2>(v, pt, sys, &ms[sys].counter, tot)) {
        MixState& M = ms[sys];
        const double sc = pair ? ldexp(1.0, 2 * pexp) : 1.0;
        M.bnorm2 = tot[0] * sc;
        M.rnorm2 = tot[1] * sc;
        M.relres = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
        M.rpair = pair ? 1 : 0;
        M.done = (M.relres <= M.tol || tot[1] == 0.0) ? 1 : 0;
        M.run = !M.done;
        if (!M.done) atomicAdd(n_active, 1);
    }
}

__global__ void __launch_bounds__(VTH) k_mix_xnorm(const double2* const* __restrict__ x64, MixState* __restrict__ ms,
                                                   Partials pt, long long n) {
    const int sys = blockIdx.y;
    const double2* X = x64[sys];
    double v[1] = {0.0};
    strided4(n, [&](long long i) { return X[i]; },
             [&](long long, const double2& x) { v[0] += x.x * x.x + x.y * x.y; });
    double tot[1];
    if (grid_sum<1>(v, pt, sys, &ms[sys].counter, tot)) {
        ms[sys].xnorm2 = tot[0];
        ms[sys].xzero = tot[0] == 0.0 ? 1 : 0;
        ms[sys].run = !ms[sys].xzero;
    }
}

__global__ void __launch_bounds__(VTH) k_mix_down(double2* const* __restrict__ r64, float2* const* __restrict__ r32,
                                                  const MixState* __restrict__ ms, long long n) {
    const int sys = blockIdx.y;
    if (ms[sys].done) return;
    const double sc = 1.0 / sqrt(ms[sys].rnorm2);
    const double2* R = r64[sys];
    float2* D = r32[sys];
    if (ms[sys].rpair) {
        // pairs at scale 2^-pexp: the high word times 2^pexp / ||r|| in FP32 (the low word is
        // below the FP32 rounding of the result)
        const float s32 = (float)(ldexp(1.0, ms[sys].pexp) * sc);
        strided4(n, [&](long long i) { return reinterpret_cast<const float4*>(R)[i]; },
                 [&](long long i, const float4& p) { D[i] = make_float2(__fmul_rn(p.x, s32), __fmul_rn(p.z, s32)); });
        return;
    }
    strided4(n, [&](long long i) { return R[i]; },
             [&](long long i, const double2& r) { D[i] = make_float2((float)(r.x * sc), (float)(r.y * sc)); });
}

__global__ void __launch_bounds__(VTH) k_mix_to_pair(const double2* const* __restrict__ x64, dfcplx* const* __restrict__ xdf,
                                                     MixState* __restrict__ ms, long long n) {
    const int sys = blockIdx.y;
    if (!ms[sys].run) return;
    // RMS of b (or of the initial x) in [2^(e-1), 2^e): the scaled entries sit near 1, far from the
    // ends of the FP32 exponent range that the double-float arithmetic shares
    const double ref = ms[sys].bnorm2 > 0.0 ? ms[sys].bnorm2 : ms[sys].xnorm2;
    int e = 0;
    if (ref > 0.0 && isfinite(ref)) frexp(sqrt(ref / (double)n), &e);
    if (blockIdx.x == 0 && threadIdx.x == 0) ms[sys].pexp = e;
    const double2* X = x64[sys];
    dfcplx* D = xdf[sys];
    strided4(n, [&](long long i) { return X[i]; },
             [&](long long i, const double2& x) {
                 dfcplx v;
                 v.x = df_split(x.x, e);
                 v.y = df_split(x.y, e);
                 D[i] = v;
             });
}

// the inner solve ended with a finite residual below the norm of its right-hand side
__device__ __forceinline__ bool inner_progress(const BcgState& I) { return isfinite(I.rnorm2) && I.rnorm2 < I.bnorm2; }

__global__ void __launch_bounds__(VTH) k_mix_up(double2* const* __restrict__ x64, float2* const* __restrict__ d32,
                                                MixState* __restrict__ ms, const BcgState* __restrict__ inner, long long n) {
    const int sys = blockIdx.y;
    if (ms[sys].done || !inner_progress(inner[sys])) return;
    const double sc = sqrt(ms[sys].rnorm2);
    double2* X = x64[sys];
    const float2* D = d32[sys];
    if (blockIdx.x == 0 && threadIdx.x == 0) ms[sys].xzero = 0;
    struct XD { double2 x; float2 d; };
    strided4(n, [&](long long i) { return XD{X[i], D[i]}; },
             [&](long long i, const XD& w) {
                 double2 x = w.x;
                 x.x += sc * (double)w.d.x;
                 x.y += sc * (double)w.d.y;
                 X[i] = x;
             });
}

// after k_mix_up: a system whose inner solve made no progress stops refining (its next inner solve
// would repeat this one exactly); the host reports it as not converged
__global__ void k_mix_stall(MixState* __restrict__ ms, const BcgState* __restrict__ inner, int nsys) {
    const int sys = blockIdx.x * blockDim.x + threadIdx.x;
    if (sys >= nsys || ms[sys].done || inner_progress(inner[sys])) return;
    ms[sys].done = 1;
    ms[sys].stalled = 1;
    ms[sys].run = 0;
}

// conj(a) . b of complex64 vectors with the inner-product accumulation of the FP32 solver kernels:
// per-block partials, summed in block order by k_dot_finish (diagnostic entry point).
__global__ void __launch_bounds__(VTH) k_dot_c64(const float2* __restrict__ a, const float2* __restrict__ b, long long n,
                                                 double* __restrict__ partial) {
    Sums<float2, 2> acc;
    strided4_sum(n, acc, [&](long long i) { return Two<float2>{a[i], b[i]}; },
                 [&](long long, const Two<float2>& w) {
                     acc_dot(acc, 0, w.a, w.b);
                 });
    double v[2];
    acc.finish(v);
    __shared__ double sh[32 * 2];
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = v[0];
        partial[2 * blockIdx.x + 1] = v[1];
    }
}
__global__ void k_dot_finish(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[2 * b + threadIdx.x];
        out[threadIdx.x] = s;
    }
}
cudaError_t launch_dot_c64(const float2* a, const float2* b, long long n, double* partial, int nblk, double* out,
                           cudaStream_t s) {
    k_dot_c64<<<nblk, VTH, 0, s>>>(a, b, n, partial);
    k_dot_finish<<<1, 32, 0, s>>>(partial, nblk, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
template <typename T>
cudaError_t bcg_init(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int x_zero,
                     const MixState* skip, int* n_active, cudaStream_t s, long long* nl) {
    k_bcg_init<T><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(vecs, st, pt, n, x_zero, skip, n_active);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
template <typename T>
cudaError_t bcg_update_p(const BcgVecs<T>* vecs, BcgState* st, long long n, int nsys, int nblk, cudaStream_t s, long long* nl) {
    k_bcg_p<T><<<dim3(nblk, nsys), VTH, 0, s>>>(vecs, st, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
template <typename T>
cudaError_t bcg_alpha(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int* n_active, cudaStream_t s,
                      long long* nl) {
    k_bcg_alpha<T><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(vecs, st, pt, n, n_active);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
template <typename T>
cudaError_t bcg_s(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, cudaStream_t s, long long* nl) {
    k_bcg_s<T><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(vecs, st, pt, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
template <typename T>
cudaError_t bcg_omega(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, cudaStream_t s, long long* nl) {
    k_bcg_omega<T><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(vecs, st, pt, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
template <typename T>
cudaError_t bcg_xr(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int* n_active, cudaStream_t s,
                   long long* nl) {
    k_bcg_xr<T><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(vecs, st, pt, n, n_active);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

// dst: mapped host memory (its device alias); one block of word stores
__global__ void __launch_bounds__(VTH) k_publish(const unsigned int* __restrict__ src, unsigned int* dst, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

cudaError_t publish(const void* src, void* dst, size_t bytes, cudaStream_t s, long long* nl) {
    k_publish<<<1, VTH, 0, s>>>(static_cast<const unsigned int*>(src), static_cast<unsigned int*>(dst),
                                (int)(bytes / sizeof(unsigned int)));
    if (nl) *nl += 1;
    return cudaGetLastError();
}

cudaError_t dot_finish(const DotSink* sinks, int nsys, cudaStream_t s, long long* nl) {
    k_dot_finish<<<nsys, VTH, 0, s>>>(sinks);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

#define LSM_INST(T)                                                                                                   \
    template cudaError_t bcg_init<T>(const BcgVecs<T>*, BcgState*, Partials, long long, int, int, const MixState*,   \
                                     int*, cudaStream_t, long long*);                                                 \
    template cudaError_t bcg_update_p<T>(const BcgVecs<T>*, BcgState*, long long, int, int, cudaStream_t, long long*); \
    template cudaError_t bcg_alpha<T>(const BcgVecs<T>*, BcgState*, Partials, long long, int, int*, cudaStream_t,     \
                                      long long*);                                                                    \
    template cudaError_t bcg_s<T>(const BcgVecs<T>*, BcgState*, Partials, long long, int, cudaStream_t, long long*);  \
    template cudaError_t bcg_omega<T>(const BcgVecs<T>*, BcgState*, Partials, long long, int, cudaStream_t, long long*); \
    template cudaError_t bcg_xr<T>(const BcgVecs<T>*, BcgState*, Partials, long long, int, int*, cudaStream_t, long long*);
LSM_INST(float)
LSM_INST(double)
#undef LSM_INST

cudaError_t mix_residual(const double2* const* b, const double2* const* ax, double2* const* r64, MixState* ms, Partials pt,
                         long long n, int nsys, int* n_active, cudaStream_t s, long long* nl, bool pair) {
    if (pair) k_mix_res<true><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(b, ax, r64, ms, pt, n, n_active);
    else k_mix_res<false><<<dim3(pt.nblk, nsys), VTH, 0, s>>>(b, ax, r64, ms, pt, n, n_active);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t mix_down(double2* const* r64, float2* const* r32, const MixState* ms, long long n, int nsys, int nblk, cudaStream_t s,
                     long long* nl) {
    k_mix_down<<<dim3(nblk, nsys), VTH, 0, s>>>(r64, r32, ms, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t mix_xnorm(const double2* const* x64, MixState* ms, Partials pt, long long n, int nsys, cudaStream_t s,
                      long long* nl) {
    k_mix_xnorm<<<dim3(pt.nblk, nsys), VTH, 0, s>>>(x64, ms, pt, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t mix_to_pair(const double2* const* x64, dfcplx* const* xdf, MixState* ms, long long n, int nsys, int nblk,
                        cudaStream_t s, long long* nl) {
    k_mix_to_pair<<<dim3(nblk, nsys), VTH, 0, s>>>(x64, xdf, ms, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t mix_up(double2* const* x64, float2* const* d32, MixState* ms, const BcgState* inner, long long n, int nsys, int nblk,
                   cudaStream_t s, long long* nl) {
    k_mix_up<<<dim3(nblk, nsys), VTH, 0, s>>>(x64, d32, ms, inner, n);
    k_mix_stall<<<(nsys + 127) / 128, 128, 0, s>>>(ms, inner, nsys);
    if (nl) *nl += 2;
    return cudaGetLastError();
}

}  // namespace lsm
