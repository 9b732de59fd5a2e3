// synth.cu - receiver time traces from frequency-domain receiver data (Sec. 4.1.2).
//
// With time dependence exp(-i w t) and a real medium, U(-f) = conj(U(f)); for frequencies
// f_k = k df, k = 0..K, the inverse Fourier integral becomes
//   u(t) = df * [ W_0 U_0 + 2 Re sum_{k>=1} W_k U_k exp(-2 pi i f_k t) ],
// W the Ricker spectrum 2 f^2 / (sqrt(pi) fp^3) exp(-f^2/fp^2) exp(+2 pi i f t0).  FP64.
#include "kernels.h"

namespace lsm {

__global__ void k_time_traces(int nf, double df, int ntr, const double2* __restrict__ U, int nt, double dt, double fp,
                              double t0, double* __restrict__ out) {
    extern __shared__ double2 sW[];   // df * weight * W_k
    for (int k = threadIdx.x; k < nf; k += blockDim.x) {
        const double f = k * df;
        const double amp = 2.0 * f * f / (sqrt(M_PI) * fp * fp * fp) * exp(-(f / fp) * (f / fp));
        double s, c;
        sincospi(2.0 * f * t0, &s, &c);
        const double wk = (k == 0 ? 1.0 : 2.0) * df * amp;
        sW[k] = make_double2(wk * c, wk * s);
    }
    __syncthreads();
    const long long total = (long long)ntr * nt;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int tr = (int)(i / nt);
        const int j = (int)(i % nt);
        const double t = j * dt;
        double acc = 0.0;
        for (int k = 0; k < nf; ++k) {
            const double2 u = U[(long long)k * ntr + tr];
            const double2 w = sW[k];
            const double2 wu = make_double2(w.x * u.x - w.y * u.y, w.x * u.y + w.y * u.x);
            double s, c;
            sincospi(-2.0 * k * df * t, &s, &c);
            acc += wu.x * c - wu.y * s;   // Re(wu * exp(-2 pi i f t))
        }
        out[i] = acc;
    }
}

cudaError_t launch_time_traces(int nf, double df, int ntr, const double2* U, int nt, double dt, double fp, double t0,
                               double* out, cudaStream_t st) {
    const long long total = (long long)ntr * nt;
    long long nb = (total + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    if (nb < 1) nb = 1;
    const size_t sm = (size_t)nf * sizeof(double2);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_time_traces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_time_traces<<<(int)nb, 256, sm, st>>>(nf, df, ntr, U, nt, dt, fp, t0, out);
    return cudaGetLastError();
}

// Receiver gather: out[r * 3 + c] = u[c * N + node[r]] for nrec receivers (node = linear index
// (iz ny + iy) nx + ix), one row of the [nf][3 nrec] spectra array of the seismogram chain.
__global__ void k_gather_receivers(const double2* __restrict__ u, long long N, const long long* __restrict__ node, int nrec,
                                   double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * nrec) return;
    const int r = i / 3, c = i - 3 * r;
    out[i] = u[(long long)c * N + node[r]];
}

cudaError_t launch_gather_receivers(const double2* u, long long N, const long long* node, int nrec, double2* out,
                                    cudaStream_t st) {
    const int n = 3 * nrec;
    k_gather_receivers<<<(n + 255) / 256, 256, 0, st>>>(u, N, node, nrec, out);
    return cudaGetLastError();
}

}  // namespace lsm
