// solver.cuh - BiCGSTAB state and launchers (internal).
#pragma once
#include "kernels.h"

namespace lsm {

// Device-resident state of one system's BiCGSTAB (Sec. 3.2; Van der Vorst 1992).  Scalars in FP64.
struct BcgState {
    double2 rho;        // <r^, r> of the current iteration
    double2 alpha;
    double2 omega;
    double2 beta;       // for the next p update
    double2 rv;         // <r^, v>
    double2 ts;         // <t, s>
    double tt;          // <t, t>
    double bnorm2;      // ||b||^2
    double tol2;        // (tol ||b||)^2
    double rnorm2;      // ||r||^2 of the last update
    double snorm2;
    int iters;
    int maxit;
    int status;         // 0 ok / running, <0 lsm_status error
    int active;         // still iterating
    int half;           // converged on the half step this iteration
    int run_v;          // apply p -> v runs
    int run_t;          // apply s -> t runs
    unsigned int counter;
};

// An inner product of the BiCGSTAB iteration folded into the epilogue of the apply that produces
// one of its operands (the inverse x pass writes out = A u): mode DOT_RV accumulates <r^, out>
// (r^ at rh) and finishes alpha; mode DOT_TS accumulates <out, u> and <out, out> and finishes
// omega.  partials: nparts x 4 floats for this system, one (Re, Im, |out|^2, 0) per epilogue
// warp; dot_finish adds them in FP64 in a fixed order into st.
enum { DOT_RV = 1, DOT_TS = 2 };
struct DotSink {
    BcgState* st;
    const void* rh;
    float* partials;
    int nparts;
    int mode;
    int* n_active;
};

template <typename T>
struct BcgVecs {
    typedef typename cplx_of<T>::type C;
    const C* b;
    C *x, *r, *rh, *p, *v, *s, *t;
};

// Refinement state of one system in the mixed-precision solve (FP64 outer residual).
struct MixState {
    double bnorm2;
    double rnorm2;
    double relres;
    double tol;
    int done;
    int run;            // FP64 residual apply runs
    int xzero;          // the iterate is exactly zero: the residual is b, no apply needed
    unsigned int counter;
    double xnorm2;      // ||x||^2 of the initial iterate
    int pexp;           // double-float residual apply: x entered scaled by 2^-pexp
    int rpair;          // the residual buffer holds double-float pairs scaled by 2^-pexp
    int stalled;        // an inner solve ended without reducing its residual: refinement stopped
};

struct Partials {
    double* buf;        // [nsys][nblk][4]
    int nblk;
};

// skip: optional per-system refinement state; systems with skip[i].done keep the state the host wrote
template <typename T>
cudaError_t bcg_init(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int x_zero,
                     const MixState* skip, int* n_active, cudaStream_t s, long long* nl);
template <typename T>
cudaError_t bcg_update_p(const BcgVecs<T>* vecs, BcgState* st, long long n, int nsys, int nblk, cudaStream_t s, long long* nl);
template <typename T>
cudaError_t bcg_alpha(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int* n_active,
                      cudaStream_t s, long long* nl);
template <typename T>
cudaError_t bcg_s(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, cudaStream_t s, long long* nl);
template <typename T>
cudaError_t bcg_omega(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, cudaStream_t s, long long* nl);
// Copy bytes (a multiple of 4) from device memory src to dst, the device alias of mapped host
// memory, with one block of stores on stream s.
cudaError_t publish(const void* src, void* dst, size_t bytes, cudaStream_t s, long long* nl);
// alpha or omega of each of nsys systems from the partial sums of its DotSink (sinks: device array)
cudaError_t dot_finish(const DotSink* sinks, int nsys, cudaStream_t s, long long* nl);
template <typename T>
cudaError_t bcg_xr(const BcgVecs<T>* vecs, BcgState* st, Partials pt, long long n, int nsys, int* n_active,
                   cudaStream_t s, long long* nl);

// mixed refinement: r64 = b - ax (relres), r32 = r64/||r64||, x64 += ||r64|| d32
// xzero = (||x||^2 == 0) per system; the FP64 residual apply is skipped for those systems
cudaError_t mix_xnorm(const double2* const* x64, MixState* ms, Partials pt, long long n, int nsys, cudaStream_t s,
                      long long* nl);
cudaError_t mix_residual(const double2* const* b, const double2* const* ax, double2* const* r64, MixState* ms,
                         Partials pt, long long n, int nsys, int* n_active, cudaStream_t s, long long* nl,
                         bool pair = false);
// x (complex128) -> double-float pairs scaled by the power of two 2^-pexp that brings the RMS of b
// (of x before b is known) near 1, recorded in ms.pexp; systems with ms.run == 0 are skipped.
// With pair, mix_residual reads A x as double-float pairs at that scale and leaves r = b - A x as
// pairs at the same scale (ms.rpair), which mix_down normalises to complex64.
cudaError_t mix_to_pair(const double2* const* x64, dfcplx* const* xdf, MixState* ms, long long n, int nsys, int nblk,
                        cudaStream_t s, long long* nl);
cudaError_t mix_down(double2* const* r64, float2* const* r32, const MixState* ms, long long n, int nsys, int nblk,
                     cudaStream_t s, long long* nl);
// x += ||r|| d for the systems whose inner solve (state inner[sys]) reduced its residual; a system
// whose inner solve did not (or ended non-finite) keeps x and is marked done and stalled.
cudaError_t mix_up(double2* const* x64, float2* const* d32, MixState* ms, const BcgState* inner, long long n, int nsys, int nblk,
                   cudaStream_t s, long long* nl);

int vec_blocks(long long n);

// conj(a) . b over n complex64 elements with the FP32 solver's inner-product accumulation;
// partial: 2 * nblk doubles of scratch, out: 2 doubles (device)
cudaError_t launch_dot_c64(const float2* a, const float2* b, long long n, double* partial, int nblk, double* out,
                           cudaStream_t s);

}  // namespace lsm
