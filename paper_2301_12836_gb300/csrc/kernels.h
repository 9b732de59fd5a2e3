// kernels.h - host-side launchers of the CUDA kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "dfloat.cuh"

namespace lsm {

// Per-system arguments of one operator application.  One entry per system of a batch;
// kernels index them with a grid dimension.  All systems of a batch share one medium.
template <typename T>
struct ApplySys {
    typedef typename cplx_of<T>::type C;
    const C* u;          // input field [3][nz][ny][nx]
    C* out;              // result [3][nz][ny][nx]
    const C* ghat;       // octant spectra [6 or 24][nz+1][ny+1][nx+1], scaled by 1/P: G (11 22 33 23 13 12),
                         // then, in the sampled-H form, H_iJ at plane 6 + 6 i + J
    C* w1;               // workspace (see apply_ws_elems)
    C* w2;               // workspace
    T omega2;            // w^2
    const int* run;      // system runs when run == nullptr or *run != 0
    unsigned long long* count;  // incremented once per executed system apply (may be nullptr)
    const void* dot = nullptr;  // BiCGSTAB iteration applies only: the DotSink (solver.cuh) whose inner
                                // product the epilogue accumulates; used when Medium::dots is set
};

// CUDA-event timing of every stage of the apply, per precision (diagnostics).  Stages: 0 stress,
// 1 div+fftx, 2 fft y forward, 3 fft z + Green multiply, 4 fft y inverse, 5 fftx inverse + epilogue.
struct KTimer {
    int on = 0;
    cudaEvent_t* ev = nullptr;   // 2 * cap events
    int* tag = nullptr;          // slot of each recorded pair: precision * 6 + stage (precision 1 = FP32)
    int cap = 0;
    int used = 0;
    int open = 0;
    double ms[12] = {0};         // flushed totals per slot
    long long launches[12] = {0};
};
void ktimer_mark(KTimer* t, int stage, bool f32, cudaStream_t st, int end);
void ktimer_flush(KTimer* t);

struct Medium {
    Dims d;
    const void* dC;      // [21][N] of T
    const void* drho;    // [N] of T
    KTimer* timer;       // optional stage timer
    int kernel;          // 0: difference form (6 spectra); 1: sampled-H form (24 spectra)
    int sched[6];        // FFT schedule variant per apply stage (0 default; see the pass launchers)
    int dots = 0;        // DOT_RV or DOT_TS: the systems' ApplySys::dot are set and the FP32 epilogue
                         // sums that inner product (only where epilogue_dots_available says so)
};

struct Plans {
    FftPlan px, py, pz;
    const void* twx;     // twiddle tables of T: exp(-2 pi i k / L)
    const void* twy;
    const void* twz;
};

// workspace elements (complex) needed by one system's apply / adjoint in w1 and w2 (kernel as in Medium)
void apply_ws_elems(const Dims& d, int kernel, long long* w1, long long* w2);

// True when the forward FP32 apply's epilogue can accumulate the BiCGSTAB inner product named by
// each system's ApplySys::dot (the warp-line inverse x pass: lengths 16, 64 and 256 with the default
// schedule), and the number of partial sums (one per epilogue warp) it writes per system.
bool epilogue_dots_available(const Medium& m);
int epilogue_dot_parts(const Dims& d);

// Operator A u (forward) or A^H u (adjoint) for nsys systems; sys is a device array.
template <typename T>
cudaError_t launch_apply(const Medium& m, const Plans& pl, const ApplySys<T>* sys_dev, int nsys,
                         cudaStream_t st, long long* nlaunch);
template <typename T>
cudaError_t launch_adjoint(const Medium& m, const Plans& pl, const ApplySys<T>* sys_dev, int nsys,
                           cudaStream_t st, long long* nlaunch);

// Contrast gradient of Re<lam, K_T(Dv dC eps(u) + w^2 drho u)>: gC [21][N], grho [N] (FP64, device);
// sys[0] supplies lam (as u), the spectrum, omega^2 and the workspaces.  accumulate adds to the outputs.
cudaError_t launch_gradient(const Medium& m, const Plans& pl, const ApplySys<double>* sys, const double2* u, double* gC,
                            double* grho, int accumulate, cudaStream_t st, long long* nl);

// Moment-tensor gradient Re<lam, d u0 / d M_J>, J = 0..5 (Voigt), summed deterministically into out[6]
// (device); partial is scratch of 6 * 4096 doubles.
cudaError_t launch_source_gradient(const Dims& d, double lam, double mu, double rho, double omega, int green,
                                   const double* xs, const double2* lamv, double* partial, double* out, cudaStream_t st,
                                   long long* nl);

// Green spectrum setup: writes the octant spectrum (double) scaled by 1/P into ghat64,
// using scratch (6 * Lx*Ly*Lz complex double).  green: 0 exact, 1 paper.  kernel 1 (sampled-H form)
// also writes the 18 octant spectra of H_iJ after the 6 of G (ghat64 then holds 24 planes).
cudaError_t launch_green_setup(const Dims& d, const Plans& pl64, double lam, double mu, double rho,
                               double omega, int green, int kernel, double2* scratch, double2* ghat64,
                               cudaStream_t st, long long* nlaunch);

// Background fields u0[m] of nm moment tensors M6[6m..6m+5] at one position (complex double);
// flag set to 1 if a node hits the source.
cudaError_t launch_source(const Dims& d, double lam, double mu, double rho, double omega, int green, int nm,
                          const double* M6, const double* xs, double2* const* u0, int* flag,
                          cudaStream_t st, long long* nlaunch);

// Absorbing-boundary weight (Eq. 25) applied in place to the 21 contrast planes and drho (FP64).
cudaError_t launch_taper(const Dims& d, int width, double* dC, double* drho, cudaStream_t st, long long* nl);

// Receiver time traces (Ricker wavelet, real-signal inverse Fourier sum), FP64.
cudaError_t launch_time_traces(int nf, double df, int ntr, const double2* U, int nt, double dt, double fp, double t0,
                               double* out, cudaStream_t st);

// Receiver gather for the seismogram chain: out[r * 3 + c] = u[c * N + node[r]], r < nrec (FP64).
cudaError_t launch_gather_receivers(const double2* u, long long N, const long long* node, int nrec, double2* out,
                                    cudaStream_t st);

// Precision converters.  d2df: n reals to double-float pairs; df2d_inplace: n double-float pairs
// to doubles in the same memory (8 bytes each).
cudaError_t launch_d2df(const double* in, dfloat* out, long long n, cudaStream_t st, long long* nlaunch);
cudaError_t launch_df2d_inplace(void* buf, long long n, cudaStream_t st, long long* nlaunch);
cudaError_t launch_d2f(const double* in, float* out, long long n, cudaStream_t st, long long* nlaunch);
cudaError_t launch_f2d_c(const float2* in, double2* out, long long n, cudaStream_t st, long long* nlaunch);

// Dynamic shared memory opt-in for the kernels (call once per device).
cudaError_t init_kernel_attributes();

}  // namespace lsm
