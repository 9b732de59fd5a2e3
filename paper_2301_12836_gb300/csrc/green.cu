// green.cu - background Green's tensor (Eq. 7, Appendix A): the sampled kernel table and the
// moment-tensor background field (Eqs. 13-16).  All FP64.
//
// Both closed forms are evaluated in radial form, G_ij(x) = f(r) d_ij + g(r) g_i g_j with
// g = x / r, so that the derivative needed by the source term is
//   dG_ij/dx_k = f'(r) g_k d_ij + g'(r) g_i g_j g_k + g(r)/r (d_ik g_j + d_jk g_i - 2 g_i g_j g_k).
//
// exact (full isotropic solution, outgoing exp(+i k r)):
//   4 pi rho f = e_b/(b^2 r) - Q,   4 pi rho g = e_a/(a^2 r) - e_b/(b^2 r) + 3 Q,
//   Q(r) = [(1 - i k_b r) e_b - (1 - i k_a r) e_a] / (w^2 r^3) = [psi(k_b r)/b^2 - psi(k_a r)/a^2] / r,
//   psi(x) = ((1 - i x) e^{ix} - 1) / x^2, evaluated by its Taylor series for |x| < 1/2 (no
//   cancellation at small w r), directly otherwise; Q' = (e_b/b^2 - e_a/a^2)/r^2 - 3 Q / r.
// paper (near field Eq. A.4 + far field Eq. A.5):
//   4 pi rho f = e_b/(b^2 r) - 4 pi rho Cn / r,  4 pi rho g = e_a/(a^2 r) - e_b/(b^2 r) + 12 pi rho Cn / r,
//   Cn = (1 - b^2/a^2) / (8 pi rho b^2).
#include "kernels.h"

namespace lsm {

constexpr int MAXM = 8;   // moment tensors per source launch

struct GreenPar {
    double a, b, rho, w;   // P, S velocities, density, angular frequency
    int mode;              // 0 exact, 1 paper
    // derived on the host (make_green_par), so that no node divides by them again
    double c4;             // 1 / (4 pi rho)
    double ka, kb;         // w / a, w / b
    double ia2, ib2;       // 1 / a^2, 1 / b^2
    double ika2, ikb2;     // 1 / ka^2, 1 / kb^2
    double cn;             // static term of the paper's near field (mode 1)
};

static GreenPar make_green_par(double lam, double mu, double rho, double omega, int green) {
    GreenPar p;
    p.a = sqrt((lam + 2.0 * mu) / rho);
    p.b = sqrt(mu / rho);
    p.rho = rho;
    p.w = omega;
    p.mode = green;
    p.c4 = 1.0 / (4.0 * M_PI * rho);
    p.ka = omega / p.a;
    p.kb = omega / p.b;
    p.ia2 = 1.0 / (p.a * p.a);
    p.ib2 = 1.0 / (p.b * p.b);
    p.ika2 = 1.0 / (p.ka * p.ka);
    p.ikb2 = 1.0 / (p.kb * p.kb);
    p.cn = (1.0 - p.b * p.b * p.ia2) / (8.0 * M_PI * rho) * p.ib2;
    return p;
}

__device__ __forceinline__ double2 cexpi(double phase) {
    double s, c;
    sincos(phase, &s, &c);
    return make_double2(c, s);
}

// psi(x) = ((1 - i x) e^{ix} - 1) / x^2 = sum_m i^m (m+1)/(m+2)! x^m; e = e^{ix} and ix2 = 1/x^2
// are supplied by the caller (it has them already)
__device__ __forceinline__ double2 psi(double x, double2 e, double ix2) {
    if (fabs(x) < 0.5) {
        // coefficients (m+1)/(m+2)! for m = 0..14
        const double a[15] = {1.0 / 2.0, 2.0 / 6.0, 3.0 / 24.0, 4.0 / 120.0, 5.0 / 720.0, 6.0 / 5040.0,
                              7.0 / 40320.0, 8.0 / 362880.0, 9.0 / 3628800.0, 10.0 / 39916800.0,
                              11.0 / 479001600.0, 12.0 / 6227020800.0, 13.0 / 87178291200.0,
                              14.0 / 1307674368000.0, 15.0 / 20922789888000.0};
        // real part: m even, sign (-1)^(m/2); imaginary: m odd, sign (-1)^((m-1)/2)
        const double x2 = x * x;
        double re = 0.0, im = 0.0;
        for (int m = 14; m >= 0; m -= 2) re = re * (-x2) + a[m];
        for (int m = 13; m >= 1; m -= 2) im = im * (-x2) + a[m];
        return make_double2(re, im * x);
    }
    return make_double2((e.x + x * e.y - 1.0) * ix2, (e.y - x * e.x) * ix2);
}

// f, g and their radial derivatives at distance r (ir = 1 / r)
__device__ void radial(const GreenPar& p, double r, double ir, double2& f, double2& g, double2& fp, double2& gp) {
    const double c4 = p.c4, ka = p.ka, kb = p.kb, ia2 = p.ia2, ib2 = p.ib2;
    const double2 ea = cexpi(ka * r), eb = cexpi(kb * r);
    // E_c = e_c / r and E_c' = (i k_c - 1/r) E_c
    const double2 Ea = make_double2(ea.x * ir, ea.y * ir);
    const double2 Eb = make_double2(eb.x * ir, eb.y * ir);
    const double2 Eap = make_double2(-ka * Ea.y - ir * Ea.x, ka * Ea.x - ir * Ea.y);
    const double2 Ebp = make_double2(-kb * Eb.y - ir * Eb.x, kb * Eb.x - ir * Eb.y);
    if (p.mode == 0) {
        const double ir2 = ir * ir;
        const double2 pa = psi(ka * r, ea, p.ika2 * ir2), pb = psi(kb * r, eb, p.ikb2 * ir2);
        const double2 Q = make_double2((pb.x * ib2 - pa.x * ia2) * ir, (pb.y * ib2 - pa.y * ia2) * ir);
        const double2 Qp = make_double2((eb.x * ib2 - ea.x * ia2) * ir * ir - 3.0 * Q.x * ir,
                                        (eb.y * ib2 - ea.y * ia2) * ir * ir - 3.0 * Q.y * ir);
        f = make_double2(c4 * (Eb.x * ib2 - Q.x), c4 * (Eb.y * ib2 - Q.y));
        g = make_double2(c4 * (Ea.x * ia2 - Eb.x * ib2 + 3.0 * Q.x), c4 * (Ea.y * ia2 - Eb.y * ib2 + 3.0 * Q.y));
        fp = make_double2(c4 * (Ebp.x * ib2 - Qp.x), c4 * (Ebp.y * ib2 - Qp.y));
        gp = make_double2(c4 * (Eap.x * ia2 - Ebp.x * ib2 + 3.0 * Qp.x), c4 * (Eap.y * ia2 - Ebp.y * ib2 + 3.0 * Qp.y));
    } else {
        const double cn = p.cn;
        f = make_double2(c4 * Eb.x * ib2 - cn * ir, c4 * Eb.y * ib2);
        g = make_double2(c4 * (Ea.x * ia2 - Eb.x * ib2) + 3.0 * cn * ir, c4 * (Ea.y * ia2 - Eb.y * ib2));
        fp = make_double2(c4 * Ebp.x * ib2 + cn * ir * ir, c4 * Ebp.y * ib2);
        gp = make_double2(c4 * (Eap.x * ia2 - Ebp.x * ib2) - 3.0 * cn * ir * ir, c4 * (Eap.y * ia2 - Ebp.y * ib2));
    }
}

// Table on the 2n-periodic grid, [6][Lz][Ly][Lx], components (11, 22, 33, 23, 13, 12):
// h^3 G(m h) for |m_a| <= n_a - 1, m != 0; self-cell value at m = 0; zero on planes m_a = n_a.
__global__ void k_green_table(Dims d, GreenPar p, double2 self, double2* __restrict__ T) {
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    const double h3 = d.h * d.h * d.h;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % d.Lx);
        const int iy = (int)((i / d.Lx) % d.Ly);
        const int iz = (int)(i / ((long long)d.Lx * d.Ly));
        double2 out[6];
        for (int c = 0; c < 6; ++c) out[c] = make_double2(0.0, 0.0);
        if (ix != d.nx && iy != d.ny && iz != d.nz) {
            const int mx = ix < d.nx ? ix : ix - d.Lx;
            const int my = iy < d.ny ? iy : iy - d.Ly;
            const int mz = iz < d.nz ? iz : iz - d.Lz;
            if (mx == 0 && my == 0 && mz == 0) {
                out[0] = out[1] = out[2] = self;
            } else {
                const double x[3] = {mx * d.h, my * d.h, mz * d.h};
                const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                const double ir = 1.0 / r;
                const double gx = x[0] * ir, gy = x[1] * ir, gz = x[2] * ir;
                double2 f, g, fp, gp;
                radial(p, r, ir, f, g, fp, gp);
                const double gg[6] = {gx * gx, gy * gy, gz * gz, gy * gz, gx * gz, gx * gy};
                for (int c = 0; c < 6; ++c) {
                    const double dd = c < 3 ? 1.0 : 0.0;
                    out[c] = make_double2(h3 * (f.x * dd + g.x * gg[c]), h3 * (f.y * dd + g.y * gg[c]));
                }
            }
        }
        for (int c = 0; c < 6; ++c) T[c * P + i] = out[c];
    }
}

// Row i of the sampled derivative kernel of Eqs. 9-10 on the 2n-periodic grid, [6][Lz][Ly][Lx]:
// entry J = (j, k) holds h^3 dG_ij/dx_k (m h) for j = k and h^3 (dG_ij/dx_k + dG_ik/dx_j)(m h) for
// j != k (the weight of the Voigt stress sigma_J in u_s,i = sum_jk dG_ij/dx_k * sigma_jk); zero at
// m = 0 (an odd kernel averages to zero over the cell) and on the planes m_a = n_a.
__global__ void k_h_table(Dims d, GreenPar p, int i, double2* __restrict__ T) {
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    const double h3 = d.h * d.h * d.h;
    const int vj[6] = {0, 1, 2, 1, 0, 0}, vk[6] = {0, 1, 2, 2, 2, 1};
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(idx % d.Lx);
        const int iy = (int)((idx / d.Lx) % d.Ly);
        const int iz = (int)(idx / ((long long)d.Lx * d.Ly));
        double2 out[6];
        for (int c = 0; c < 6; ++c) out[c] = make_double2(0.0, 0.0);
        const int mx = ix < d.nx ? ix : ix - d.Lx;
        const int my = iy < d.ny ? iy : iy - d.Ly;
        const int mz = iz < d.nz ? iz : iz - d.Lz;
        if (ix != d.nx && iy != d.ny && iz != d.nz && (mx != 0 || my != 0 || mz != 0)) {
            const double x[3] = {mx * d.h, my * d.h, mz * d.h};
            const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            const double ir = 1.0 / r;
            const double c[3] = {x[0] * ir, x[1] * ir, x[2] * ir};
            double2 f, g, fp, gp;
            radial(p, r, ir, f, g, fp, gp);
            // dG_ij/dx_k = f' c_k d_ij + g' c_i c_j c_k + (g / r)(d_ik c_j + d_jk c_i - 2 c_i c_j c_k)
            auto dG = [&](int a, int b, int k) -> double2 {
                const double dab = a == b ? 1.0 : 0.0, dak = a == k ? 1.0 : 0.0, dbk = b == k ? 1.0 : 0.0;
                const double t1 = c[k] * dab, t2 = c[a] * c[b] * c[k];
                const double t3 = (dak * c[b] + dbk * c[a] - 2.0 * t2) * ir;
                return make_double2(fp.x * t1 + gp.x * t2 + g.x * t3, fp.y * t1 + gp.y * t2 + g.y * t3);
            };
            for (int J = 0; J < 6; ++J) {
                double2 v = dG(i, vj[J], vk[J]);
                if (vj[J] != vk[J]) {
                    const double2 w = dG(i, vk[J], vj[J]);
                    v.x += w.x;
                    v.y += w.y;
                }
                out[J] = make_double2(h3 * v.x, h3 * v.y);
            }
        }
        for (int J = 0; J < 6; ++J) T[J * P + idx] = out[J];
    }
}

// u0_i = -sum_jk M_jk dG_ij/dx_k (x - s)
//      = -[(f' + g/r) (M g)_i + (g' - 2 g/r)(g.M g) g_i + (g/r) tr(M) g_i]
// for up to MAXM moment tensors at one source position: the radial factors (the transcendental
// part) are evaluated once per node and contracted with every tensor of the set.
struct MomentSet {
    int nm;
    double M[MAXM][6];       // Voigt 11, 22, 33, 23, 13, 12
    double2* u0[MAXM];
};

__global__ void k_source(Dims d, GreenPar p, MomentSet ms, double sx, double sy, double sz, int* __restrict__ flag) {
    const long long N = d.N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % d.nx);
        const int iy = (int)((i / d.nx) % d.ny);
        const int iz = (int)(i / ((long long)d.nx * d.ny));
        const double x = ix * d.h - sx, y = iy * d.h - sy, z = iz * d.h - sz;
        const double r = sqrt(x * x + y * y + z * z);
        if (r == 0.0) {
            for (int m = 0; m < ms.nm; ++m)
                for (int c = 0; c < 3; ++c) ms.u0[m][c * N + i] = make_double2(0.0, 0.0);
            atomicExch(flag, 1);
            continue;
        }
        const double ir = 1.0 / r;
        const double g[3] = {x * ir, y * ir, z * ir};
        double2 f, gg, fp, gp;
        radial(p, r, ir, f, gg, fp, gp);
        const double2 A = make_double2(fp.x + gg.x * ir, fp.y + gg.y * ir);
        const double2 B = make_double2(gp.x - 2.0 * gg.x * ir, gp.y - 2.0 * gg.y * ir);
        const double2 Cc = make_double2(gg.x * ir, gg.y * ir);
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
            if (m >= ms.nm) break;
            const double* M = ms.M[m];   // 11 22 33 23 13 12
            const double Mg[3] = {M[0] * g[0] + M[5] * g[1] + M[4] * g[2],
                                  M[5] * g[0] + M[1] * g[1] + M[3] * g[2],
                                  M[4] * g[0] + M[3] * g[1] + M[2] * g[2]};
            const double gMg = g[0] * Mg[0] + g[1] * Mg[1] + g[2] * Mg[2];
            const double tr = M[0] + M[1] + M[2];
            // u0_c = -(A (M g)_c + (B g.M.g + C tr M) g_c): the g_c terms share one coefficient
            const double2 D = make_double2(B.x * gMg + Cc.x * tr, B.y * gMg + Cc.y * tr);
            for (int c = 0; c < 3; ++c)
                ms.u0[m][c * N + i] = make_double2(-(A.x * Mg[c] + D.x * g[c]), -(A.y * Mg[c] + D.y * g[c]));
        }
    }
}

// Re<lam, d u0/d M_J> for the unit Voigt moments e_J (M23 = M32 = 1 for J = 3, and so on):
// u0_i(e_J) = -[(f' + g/r) (E_J g)_i + (g' - 2 g/r)(g.E_J g) g_i + (g/r) tr(E_J) g_i].
// Block b writes its six partial sums to partial[b * 6 + J]; k_sum6 adds them in block order.
constexpr int SG_BLOCKS = 4096;
__global__ void __launch_bounds__(256) k_source_grad(Dims d, GreenPar p, double sx, double sy, double sz,
                                                     const double2* __restrict__ lamv, double* __restrict__ partial) {
    const long long N = d.N;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % d.nx);
        const int iy = (int)((i / d.nx) % d.ny);
        const int iz = (int)(i / ((long long)d.nx * d.ny));
        const double x = ix * d.h - sx, y = iy * d.h - sy, z = iz * d.h - sz;
        const double r = sqrt(x * x + y * y + z * z);
        if (r == 0.0) continue;  // u0 is zero on a node that coincides with the source
        const double ir = 1.0 / r;
        const double g[3] = {x * ir, y * ir, z * ir};
        double2 f, gg, fp, gp;
        radial(p, r, ir, f, gg, fp, gp);
        const double2 A = make_double2(fp.x + gg.x * ir, fp.y + gg.y * ir);
        const double2 B = make_double2(gp.x - 2.0 * gg.x * ir, gp.y - 2.0 * gg.y * ir);
        const double2 Cc = make_double2(gg.x * ir, gg.y * ir);
        double2 l[3];
        for (int c = 0; c < 3; ++c) l[c] = lamv[c * N + i];
        // Voigt pairs of e_J: 11, 22, 33, 23, 13, 12
        const int pa[6] = {0, 1, 2, 1, 0, 0}, pb[6] = {0, 1, 2, 2, 2, 1};
        for (int J = 0; J < 6; ++J) {
            double Mg[3] = {0, 0, 0};
            Mg[pa[J]] += g[pb[J]];
            if (pa[J] != pb[J]) Mg[pb[J]] += g[pa[J]];
            const double gMg = g[0] * Mg[0] + g[1] * Mg[1] + g[2] * Mg[2];
            const double tr = J < 3 ? 1.0 : 0.0;
            double s = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double s1 = Mg[c], s2 = gMg * g[c], s3 = tr * g[c];
                const double ux = -(A.x * s1 + B.x * s2 + Cc.x * s3), uy = -(A.y * s1 + B.y * s2 + Cc.y * s3);
                s += l[c].x * ux + l[c].y * uy;   // Re(conj(lam) u0)
            }
            acc[J] += s;
        }
    }
    __shared__ double sh[6][256];
    for (int J = 0; J < 6; ++J) sh[J][threadIdx.x] = acc[J];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int J = 0; J < 6; ++J) sh[J][threadIdx.x] += sh[J][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int J = 0; J < 6; ++J) partial[blockIdx.x * 6 + J] = sh[J][0];
}

__global__ void k_sum6(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[b * 6 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

static inline int gsz(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t fft3_inplace_setup(const Dims& d, const Plans& pl, double2* buf, int ncomp, cudaStream_t st, long long* nl);
cudaError_t launch_extract_octant(const Dims& d, const double2* full, double2* oct, double scale, cudaStream_t st, long long* nl);

cudaError_t launch_green_setup(const Dims& d, const Plans& pl64, double lam, double mu, double rho, double omega,
                               int green, int kernel, double2* scratch, double2* ghat64, cudaStream_t st, long long* nl) {
    const GreenPar p = make_green_par(lam, mu, rho, omega, green);
    // cell average of G over [-h/2, h/2]^3 times h^3, to O(w h): the static Kelvin part gives
    // (1/(3a^2) + 2/(3b^2)) C h^2 / (4 pi rho) with C = int_{unit cube} dV/|x| = 3 ln(2+sqrt3) - pi/2,
    // the r^0 term of the expansion gives i w h^3 (1/(3a^3) + 2/(3b^3)) / (4 pi rho).
    const double Cself = 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * M_PI;
    const double c4 = 1.0 / (4.0 * M_PI * rho);
    const double h = d.h;
    double2 self;
    self.x = c4 * (1.0 / (3.0 * p.a * p.a) + 2.0 / (3.0 * p.b * p.b)) * Cself * h * h;
    self.y = c4 * omega * (1.0 / (3.0 * p.a * p.a * p.a) + 2.0 / (3.0 * p.b * p.b * p.b)) * h * h * h;
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    k_green_table<<<gsz(P), 256, 0, st>>>(d, p, self, scratch);
    if (nl) *nl += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = fft3_inplace_setup(d, pl64, scratch, 6, st, nl);
    if (e != cudaSuccess) return e;
    e = launch_extract_octant(d, scratch, ghat64, 1.0 / (double)P, st, nl);
    if (e != cudaSuccess || kernel != 1) return e;
    // sampled-H form: the three rows of H_iJ, six planes each, through the same scratch
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    for (int i = 0; i < 3; ++i) {
        k_h_table<<<gsz(P), 256, 0, st>>>(d, p, i, scratch);
        if (nl) *nl += 1;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = fft3_inplace_setup(d, pl64, scratch, 6, st, nl);
        if (e == cudaSuccess) e = launch_extract_octant(d, scratch, ghat64 + (6 + 6 * i) * NO, 1.0 / (double)P, st, nl);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_source(const Dims& d, double lam, double mu, double rho, double omega, int green, int nm,
                          const double* M6, const double* xs, double2* const* u0, int* flag, cudaStream_t st, long long* nl) {
    const GreenPar p = make_green_par(lam, mu, rho, omega, green);
    for (int m0 = 0; m0 < nm; m0 += MAXM) {
        MomentSet ms;
        ms.nm = nm - m0 < MAXM ? nm - m0 : MAXM;
        for (int m = 0; m < ms.nm; ++m) {
            for (int k = 0; k < 6; ++k) ms.M[m][k] = M6[6 * (m0 + m) + k];
            ms.u0[m] = u0[m0 + m];
        }
        k_source<<<gsz(d.N), 256, 0, st>>>(d, p, ms, xs[0], xs[1], xs[2], flag);
        if (nl) *nl += 1;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_source_gradient(const Dims& d, double lam, double mu, double rho, double omega, int green,
                                   const double* xs, const double2* lamv, double* partial, double* out, cudaStream_t st,
                                   long long* nl) {
    const GreenPar p = make_green_par(lam, mu, rho, omega, green);
    long long nb = (d.N + 255) / 256;
    if (nb > SG_BLOCKS) nb = SG_BLOCKS;
    if (nb < 1) nb = 1;
    k_source_grad<<<(int)nb, 256, 0, st>>>(d, p, xs[0], xs[1], xs[2], lamv, partial);
    k_sum6<<<1, 32, 0, st>>>(partial, (int)nb, out);
    if (nl) *nl += 2;
    return cudaGetLastError();
}

// Eq. 25: inside a layer of `width` nodes each axis contributes 1 - exp(-l^2 / (N h^2)), l the
// distance to the outer node plane along that axis, N the nodes along it.
__device__ __forceinline__ double taper_factor(int k, int N, double h, int width) {
    const int dist = k < N - 1 - k ? k : N - 1 - k;
    if (dist >= width) return 1.0;
    const double l = dist * h;
    return 1.0 - exp(-l * l / ((double)N * h * h));
}

__global__ void k_taper(Dims d, int width, double* __restrict__ dC, double* __restrict__ drho) {
    const long long N = d.N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % d.nx);
        const int iy = (int)((i / d.nx) % d.ny);
        const int iz = (int)(i / ((long long)d.nx * d.ny));
        const double w = taper_factor(ix, d.nx, d.h, width) * taper_factor(iy, d.ny, d.h, width) *
                         taper_factor(iz, d.nz, d.h, width);
        if (w == 1.0) continue;
        for (int k = 0; k < 21; ++k) dC[k * N + i] *= w;
        drho[i] *= w;
    }
}

cudaError_t launch_taper(const Dims& d, int width, double* dC, double* drho, cudaStream_t st, long long* nl) {
    if (width <= 0) return cudaSuccess;
    k_taper<<<gsz(d.N), 256, 0, st>>>(d, width, dC, drho);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void k_f2d_c(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

// double -> double-float: hi = fl32(v), lo = fl32(v - hi); |lo| <= ulp(hi) / 2
__global__ void k_d2df(const double* __restrict__ in, dfloat* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = in[i];
        const float h = __double2float_rn(v);
        out[i] = dfloat(h, __double2float_rn(v - (double)h));
    }
}
// double-float -> double in place (hi + lo rounded once to FP64)
__global__ void k_df2d(double* buf, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = reinterpret_cast<const float2*>(buf)[i];
        buf[i] = (double)v.x + (double)v.y;
    }
}

cudaError_t launch_d2df(const double* in, dfloat* out, long long n, cudaStream_t st, long long* nl) {
    k_d2df<<<gsz(n), 256, 0, st>>>(in, out, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t launch_df2d_inplace(void* buf, long long n, cudaStream_t st, long long* nl) {
    k_df2d<<<gsz(n), 256, 0, st>>>((double*)buf, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

cudaError_t launch_d2f(const double* in, float* out, long long n, cudaStream_t st, long long* nl) {
    k_d2f<<<gsz(n), 256, 0, st>>>(in, out, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}
cudaError_t launch_f2d_c(const float2* in, double2* out, long long n, cudaStream_t st, long long* nl) {
    k_f2d_c<<<gsz(n), 256, 0, st>>>(in, out, n);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

}  // namespace lsm
