// apply.cu - the matrix-free Lippmann-Schwinger operator (Eqs. 8, 11, 18-21) and its adjoint.
//
// One application A u = u - crop( G * q ), q_j = sum_k D_k sigma_jk + w^2 drho u_j, runs as:
//   k_stress      eps (Eq. 18, one-sided on boundary nodes) -> sigma_J = dC_JK eps_K (Eq. 11)
//   k_divq        q on the extended nodes [-1, n] (central-difference divergence of sigma plus
//                 the density term)
//   k(4)_rows     q zero-padded to 2 n_x and FFT'd along x
//   k(4)_strided  forward FFT along y (zero padding pruned on load)
//   k(4)_fftz_green  forward FFT along z, u-hat_i = sum_j G-hat_ij q-hat_j, inverse FFT along z, crop
//   k(4)_strided  inverse FFT along y, crop
//   k(4)_fftx_out inverse FFT along x, crop, Au = u - u_s
// Power-of-two line lengths 16..512 use the compile-time four-step FFT kernels (k4_*), any other
// length the runtime mixed-radix Stockham kernels.
// Only three displacement-like components pass through the FFTs: the derivative of the
// Green tensor in Eq. 8 is applied as the central difference D_k in real space, which is
// exactly the factor i sin(k h)/h of the spectral form.  The contrast source q is shifted by
// one node (index p holds node p - 1) so that it occupies [0, n+2) of the 2n-periodic grid;
// the result is then read at indices 1..n.  1/P of the inverse FFT is folded into G-hat.
#include <mutex>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "fft.cuh"
#include "fft4.cuh"
#include "solver.cuh"   // DotSink

namespace lsm {

static constexpr int NTH = 256;

// FFT engines.  GenericFFT: runtime mixed-radix Stockham plan, ping-pong buffers, any block size.
// FourStepFFT<A, B>: compile-time L = A * B, in place, exactly NL * TPL threads per block.
// Launch bounds of the FFT kernels.  Four-step tiles have at most 384 threads (FP32) or 192
// (FP64); asking for two resident FP32 blocks keeps those kernels at <= 85 registers, while the
// FP64 ones keep their 16-point DFTs in up to 255 registers without spilling.
template <typename T, bool INPLACE> struct FftBounds {
    static constexpr int threads = INPLACE ? (sizeof(T) == 8 ? 192 : 384) : 512;
    static constexpr int blocks = (INPLACE && sizeof(T) == 4) ? 2 : 1;
};
#define LSM_COMMA ,
#define LSM_FFT_BOUND(T, F) __launch_bounds__(FftBounds<T LSM_COMMA F::INPLACE>::threads, FftBounds<T LSM_COMMA F::INPLACE>::blocks)

struct GenericFFT {
    static constexpr bool INPLACE = false;
    static constexpr int TPL = 0;
    static constexpr int A_ = 0, B_ = 0;
    template <int S, typename C>
    static __device__ __forceinline__ C* run(C* a, C* b, const FftPlan& p, int NL, int LD, const C* __restrict__ tw) {
        return fft_smem<S>(a, b, p, NL, LD, tw, threadIdx.x, blockDim.x);
    }
};
template <int A, int B>
struct FourStepFFT {
    static constexpr int A_ = A, B_ = B;
    static constexpr bool INPLACE = true;
    static constexpr int TPL = FourStep<A, B>::TPL;
    template <int S, typename C>
    static __device__ __forceinline__ C* run(C* a, C*, const FftPlan&, int NL, int LD, const C* __restrict__ tw) {
        fft4_smem<A, B, S>(a, NL, LD, tw, threadIdx.x);
        return a;
    }
};

// Voigt index (order 11, 22, 33, 23, 13, 12) of the tensor pair (j, k).
__device__ __forceinline__ int t2v(int j, int k) { return (j == k) ? j : (6 - j - k); }

// index of Voigt (I, J), I <= J, in the 21 packed planes (upper triangle, row-major)
__host__ __device__ __forceinline__ int p21(int I, int J) {
    if (I > J) { int t = I; I = J; J = t; }
    return I * 6 - (I * (I - 1)) / 2 + (J - I);
}

template <typename C>
__device__ __forceinline__ void ghat_at(const C* __restrict__ g, const Dims& d, int kx, int ky, int kz,
                                        bool conj, C G[6]) {
    typedef typename real_of<C>::type T;
    const int fx = kx <= d.nx ? kx : d.Lx - kx;
    const int fy = ky <= d.ny ? ky : d.Ly - ky;
    const int fz = kz <= d.nz ? kz : d.Lz - kz;
    const T sx = kx > d.nx ? (T)-1 : (T)1;
    const T sy = ky > d.ny ? (T)-1 : (T)1;
    const T sz = kz > d.nz ? (T)-1 : (T)1;
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long i = ((long long)fz * (d.ny + 1) + fy) * (d.nx + 1) + fx;
    G[0] = __ldg(&g[i]);
    G[1] = __ldg(&g[NO + i]);
    G[2] = __ldg(&g[2 * NO + i]);
    G[3] = cscale(__ldg(&g[3 * NO + i]), sy * sz);
    G[4] = cscale(__ldg(&g[4 * NO + i]), sx * sz);
    G[5] = cscale(__ldg(&g[5 * NO + i]), sx * sy);
    if (conj) {
#pragma unroll
        for (int c = 0; c < 6; ++c) G[c] = cconj(G[c]);
    }
}

// ---------------------------------------------------------------------------------------------
// strain + contraction
// ---------------------------------------------------------------------------------------------
// Contrast stress at one model node (Eqs. 18 and 11): Voigt strain from central differences
// (one-sided on the first and last node of an axis), contracted with the 21 contrast planes.
// FP64 (arithmetic-bound) takes the differences without branches: the neighbour offsets collapse
// to the node itself at the ends, where the step is h instead of 2h, so all loads issue together;
// FP32 (memory-bound) measured faster with the ends as branches.  Same arithmetic either way.
// FP64 runs 2 blocks of 256 threads per SM (124 registers): 458 -> 406 us per system apply at
// 128^3 against 1 block (149 registers).
template <typename T>
__device__ __forceinline__ void stress_at(const Dims& d, const T* __restrict__ dC, const typename cplx_of<T>::type* __restrict__ u,
                                          long long idx, int ix, int iy, int iz, typename cplx_of<T>::type (&sg)[6]) {
    typedef typename cplx_of<T>::type C;
    const long long N = d.N;
    const long long sxy = (long long)d.nx * d.ny;
    const T ih = (T)(1.0 / d.h), i2h = (T)(0.5 / d.h);
    auto der = [&](int c, int a) -> C {
        const C* f = u + c * N;
        const int i = a == 0 ? ix : (a == 1 ? iy : iz);
        const int n = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
        const long long s = a == 0 ? 1 : (a == 1 ? (long long)d.nx : sxy);
        if constexpr (sizeof(T) == 8) {
            const long long op = i < n - 1 ? s : 0, om = i > 0 ? s : 0;
            return cscale(csub(f[idx + op], f[idx - om]), (op != 0 && om != 0) ? i2h : ih);
        } else {
            if (i == 0) return cscale(csub(f[idx + s], f[idx]), ih);
            if (i == n - 1) return cscale(csub(f[idx], f[idx - s]), ih);
            return cscale(csub(f[idx + s], f[idx - s]), i2h);
        }
    };
    C e[6];
    e[0] = der(0, 0);
    e[1] = der(1, 1);
    e[2] = der(2, 2);
    e[3] = cadd(der(1, 2), der(2, 1));
    e[4] = cadd(der(0, 2), der(2, 0));
    e[5] = cadd(der(0, 1), der(1, 0));
    T c21[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) c21[k] = __ldg(&dC[k * N + idx]);
#pragma unroll
    for (int J = 0; J < 6; ++J) {
        C s = czero<C>();
#pragma unroll
        for (int K = 0; K < 6; ++K) {
            const T c = c21[p21(J, K)];
            s.x += c * e[K].x;
            s.y += c * e[K].y;
        }
        sg[J] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 ? 8 : 2) k_stress(Dims d, const T* __restrict__ dC, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const C* __restrict__ u = S.u;
    C* __restrict__ sig = S.w1;
    const long long N = d.N;
    const long long sxy = (long long)d.nx * d.ny;
    for (long long idx = (long long)blockIdx.x * NTH + threadIdx.x; idx < N; idx += (long long)gridDim.x * NTH) {
        const int ix = (int)(idx % d.nx);
        const int iy = (int)((idx / d.nx) % d.ny);
        const int iz = (int)(idx / sxy);
        C sg[6];
        stress_at<T>(d, dC, u, idx, ix, iy, iz, sg);
#pragma unroll
        for (int J = 0; J < 6; ++J) sig[J * N + idx] = sg[J];
    }
}

// Contrast contraction fused with the divergence (Eqs. 18, 11, 8): q on the extended nodes
// [-1, n]^3, [3][ez][ey][ex] in w2, with no stress round trip through memory.  A block owns a
// TX x TY tile of extended (x, y) columns and marches through ZC extended z planes
// (blockIdx.z = chunk + chunks * system); the stress of three consecutive planes (the tile plus a
// one-node x/y halo, zero off the model) sits in a shared-memory ring, each plane computed once
// per tile and chunk (x/y halo nodes by both neighbouring tiles, the two planes before a chunk
// by both neighbouring chunks).  The arithmetic per q entry is that of k_stress + k_divq, in the
// same order.
template <typename T, int TX, int TY, int ZC>
__global__ void __launch_bounds__(TX * TY) k_sdq(Dims d, const T* __restrict__ dC, const T* __restrict__ drho,
                                                 const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY, NT = TX * TY;
    extern __shared__ unsigned char smem_raw[];
    C* ring = reinterpret_cast<C*>(smem_raw);   // [3 planes][6 comps][HP]
    const int chunks = (d.ez + ZC - 1) / ZC;
    const int chunk = blockIdx.z % chunks;
    const ApplySys<T> S = sys[blockIdx.z / chunks];
    if (S.run && !*S.run) return;
    const C* __restrict__ u = S.u;
    C* __restrict__ q = S.w2;
    const long long N = d.N;
    const long long E = (long long)d.ex * d.ey * d.ez;
    const long long sxy = (long long)d.nx * d.ny;
    const T i2h = (T)(0.5 / d.h);
    const int pz0 = chunk * ZC - 1;                                  // first model plane of the chunk
    const int pz1 = pz0 + ZC - 1 < d.nz ? pz0 + ZC - 1 : d.nz;       // last
    const int x0 = blockIdx.x * TX - 1, y0 = blockIdx.y * TY - 1;   // model coordinates of the tile's first column
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int px = x0 + tx, py = y0 + ty;                           // this thread's column, in [-1, n]
    const bool col_ok = px <= d.nx && py <= d.ny;
    const bool in_xy = px >= 0 && px < d.nx && py >= 0 && py < d.ny;
    // stress of model plane z on the halo tile into ring slot (z + 3) % 3
    auto plane = [&](int z) {
        C* R = ring + ((z + 3) % 3) * 6 * HP;
        for (int i = threadIdx.x; i < HP; i += NT) {
            const int mx = x0 - 1 + i % HX, my = y0 - 1 + i / HX;
            C sg[6];
            if (z >= 0 && z < d.nz && mx >= 0 && mx < d.nx && my >= 0 && my < d.ny) {
                stress_at<T>(d, dC, u, (long long)z * sxy + (long long)my * d.nx + mx, mx, my, z, sg);
            } else {
#pragma unroll
                for (int J = 0; J < 6; ++J) sg[J] = czero<C>();
            }
#pragma unroll
            for (int J = 0; J < 6; ++J) R[J * HP + i] = sg[J];
        }
    };
    plane(pz0 - 1);
    plane(pz0);
    const int c0 = (ty + 1) * HX + (tx + 1);   // this column in the halo tile
    for (int pz = pz0; pz <= pz1; ++pz) {
        plane(pz + 1);
        __syncthreads();
        if (col_ok) {
            const C* Rm = ring + ((pz + 2) % 3) * 6 * HP;   // plane pz - 1
            const C* Rc = ring + ((pz + 3) % 3) * 6 * HP;   // plane pz
            const C* Rp = ring + ((pz + 4) % 3) * 6 * HP;   // plane pz + 1
            C qj[3] = {czero<C>(), czero<C>(), czero<C>()};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int vx = t2v(j, 0);
                qj[j] = cadd(qj[j], csub(Rc[vx * HP + c0 + 1], Rc[vx * HP + c0 - 1]));
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int vy = t2v(j, 1);
                qj[j] = cadd(qj[j], csub(Rc[vy * HP + c0 + HX], Rc[vy * HP + c0 - HX]));
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int vz = t2v(j, 2);
                qj[j] = cadd(qj[j], csub(Rp[vz * HP + c0], Rm[vz * HP + c0]));
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) qj[j] = cscale(qj[j], i2h);
            if (in_xy && pz >= 0 && pz < d.nz) {
                const long long base = (long long)pz * sxy + (long long)py * d.nx + px;
                const T w = S.omega2 * __ldg(&drho[base]);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const C uj = u[j * N + base];
                    qj[j].x += w * uj.x;
                    qj[j].y += w * uj.y;
                }
            }
            const long long eidx = ((long long)(pz + 1) * d.ey + (py + 1)) * d.ex + (px + 1);
#pragma unroll
            for (int j = 0; j < 3; ++j) q[j * E + eidx] = qj[j];
        }
        __syncthreads();   // the next plane overwrites the ring slot of plane pz - 1
    }
}

// ---------------------------------------------------------------------------------------------
// generic strided pass: TX consecutive lines (along x) of a strided axis.  Element e of line x of
// outer (oy = blockIdx.y, comp c) lives at base + c*os2 + oy*os1 + e*es + x.
// ---------------------------------------------------------------------------------------------
struct StridedArgs {
    int nlines;        // lines along x (row length of src and dst)
    int TX;
    int in_count, in_off, out_count, out_off;
    long long src_es, src_os1, src_os2;
    long long dst_es, dst_os1, dst_os2;
    int ncomp;         // comps per system (blockIdx.z = c + ncomp * sys)
    int src_sel, dst_sel;  // 0 u, 1 out, 2 w1, 3 w2
};

template <typename C>
__device__ __forceinline__ C* pick(const ApplySys<typename real_of<C>::type>& S, int sel) {
    switch (sel) {
        case 0: return const_cast<C*>(S.u);
        case 1: return S.out;
        case 2: return S.w1;
        default: return S.w2;
    }
}

template <int DIR, class F, typename C>
__device__ __forceinline__ void strided_tile(const C* src, C* dst, const FftPlan& p, const C* __restrict__ tw,
                                             const StridedArgs& a, int x0, C* sa, C* sb) {
    const int L = p.L, TX = a.TX;
    for (int i = threadIdx.x; i < L * TX; i += blockDim.x) {
        const int l = i % TX;
        const int e = i / TX;
        const int x = x0 + l;
        const int es = e - a.in_off;
        C v = czero<C>();
        if (x < a.nlines && es >= 0 && es < a.in_count) v = src[es * a.src_es + x];
        sa[i] = v;
    }
    __syncthreads();
    C* r = F::template run<DIR>(sa, sb, p, TX, TX, tw);
    for (int i = threadIdx.x; i < a.out_count * TX; i += blockDim.x) {
        const int l = i % TX;
        const int eo = i / TX;
        const int x = x0 + l;
        if (x < a.nlines) dst[eo * a.dst_es + x] = r[(eo + a.out_off) * TX + l];
    }
}

template <typename T, int DIR, class F>
__global__ void LSM_FFT_BOUND(T, F) k_strided(FftPlan p, const typename cplx_of<T>::type* __restrict__ tw,
                                                 StridedArgs a, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    const int c = blockIdx.z % a.ncomp;
    const int s = blockIdx.z / a.ncomp;
    const ApplySys<T> S = sys[s];
    if (S.run && !*S.run) return;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = F::INPLACE ? sa : sa + (size_t)p.L * a.TX;
    const C* src = pick<C>(S, a.src_sel) + c * a.src_os2 + blockIdx.y * a.src_os1;
    C* dst = pick<C>(S, a.dst_sel) + c * a.dst_os2 + blockIdx.y * a.dst_os1;
    strided_tile<DIR, F>(src, dst, p, tw, a, blockIdx.x * a.TX, sa, sb);
}

// raw-pointer variant for the Green spectrum setup (in place allowed: each CTA owns its tile)
template <typename T, int DIR>
__global__ void __launch_bounds__(NTH) k_strided_raw(FftPlan p, const typename cplx_of<T>::type* __restrict__ tw,
                                                     StridedArgs a, const typename cplx_of<T>::type* src0,
                                                     typename cplx_of<T>::type* dst0) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = sa + (size_t)p.L * a.TX;
    const C* src = src0 + blockIdx.z * a.src_os2 + blockIdx.y * a.src_os1;
    C* dst = dst0 + blockIdx.z * a.dst_os2 + blockIdx.y * a.dst_os1;
    strided_tile<DIR, GenericFFT>(src, dst, p, tw, a, blockIdx.x * a.TX, sa, sb);
}

// four-step strided pass: step 1 loads straight from global memory, the last step stores straight
// to global memory; one shared-memory exchange in between.  Block = TX * TPL threads, line l = lx.
template <typename T, int DIR, int A, int B, int TX>
__global__ void __launch_bounds__(TX * FourStep<A LSM_COMMA B>::TPL, 4) k4_strided(const typename cplx_of<T>::type* __restrict__ tw,
                                                                     StridedArgs a, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    const int c = blockIdx.z % a.ncomp;
    const int sidx = blockIdx.z / a.ncomp;
    const ApplySys<T> S = sys[sidx];
    if (S.run && !*S.run) return;
    C* s = reinterpret_cast<C*>(smem_raw);
    const int x = blockIdx.x * TX + threadIdx.x % TX;   // this thread's line
    const bool xin = x < a.nlines;
    const C* __restrict__ src = pick<C>(S, a.src_sel) + c * a.src_os2 + blockIdx.y * a.src_os1 + x;
    C* __restrict__ dst = pick<C>(S, a.dst_sel) + c * a.dst_os2 + blockIdx.y * a.dst_os1 + x;
    const int ses = (int)a.src_es, des = (int)a.dst_es;
    const int in_off = a.in_off, in_count = a.in_count, out_off = a.out_off, out_count = a.out_count;
    auto ld = [&](int, int e) -> C {
        const int es = e - in_off;
        return (xin && es >= 0 && es < in_count) ? src[es * ses] : czero<C>();
    };
    auto st = [&](int, int k, C v) {
        const int eo = k - out_off;
        if (xin && eo >= 0 && eo < out_count) dst[eo * des] = v;
    };
    // zero padding (forward) and cropping (inverse) pruned: at most A/2 + 1 nonzero step-1 inputs,
    // at most B/2 + 1 wanted step-2 outputs per DFT (the launcher checks the line's extents)
    fft4_io<A, B, DIR, false, false, TX, (DIR < 0 ? A / 2 + 1 : A), (DIR > 0 ? B / 2 + 1 : B)>(s, tw, threadIdx.x, ld, st);
}

// four-step z pass with the Green multiply.  Block = 3 TX * TPL threads; line l = c * TX + lx.
// One block serves one (kx tile, ky) column for every system of the batch in turn.  Its slice of
// the octant spectrum (|kz| = 0..nz, 6 components, TX values of kx at one ky) is copied to shared
// memory asynchronously, once for all consecutive systems that share the spectrum (the sources
// of one frequency), while the first of them runs its forward FFT.
template <typename T, bool CONJ, int A, int B, int TX>
__global__ void __launch_bounds__(3 * TX * FourStep<A LSM_COMMA B>::TPL, 2) k4_fftz_green(
    Dims d, const typename cplx_of<T>::type* __restrict__ tw, const ApplySys<T>* __restrict__ sys, int nsys, int in_count,
    int in_off, int out_count, int out_off, int src_sel, int dst_sel) {
    typedef typename cplx_of<T>::type C;
    typedef typename real_of<C>::type R;
    constexpr int NL = 3 * TX;
    constexpr int L = A * B;
    constexpr int E = (int)(128 / sizeof(C));
    // spectrum slice [nz+1][6][TX] with row stride GS: consecutive kz rows start TX elements
    // apart modulo a 128-byte bank row, so the multiply's reads are conflict-free
    constexpr int GS = 6 * TX + (((TX - 6 * TX) % E) + E) % E;
    constexpr int YB = B * fft4_ystride<A, C>(NL);
    extern __shared__ unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* sG = s + (YB > L * NL ? YB : L * NL);
    const int ky = blockIdx.y;
    const int x0 = blockIdx.x * TX;
    const int fy = ky <= d.ny ? ky : d.Ly - ky;
    const unsigned my = ky > d.ny ? SIGN_BIT : 0u;
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const int plane = d.Ly * d.Lx;
    // this thread's line (fixed through both FFTs): component cl, column x0 + lxl
    const int lt = threadIdx.x % NL;
    const int cl = lt / TX, lxl = lt - cl * TX;
    const bool xin = x0 + lxl < d.Lx;
    const long long col = (long long)ky * d.Lx + x0 + lxl;
    const C* staged = nullptr;
    for (int si = 0; si < nsys; ++si) {
        const ApplySys<T> S = sys[si];
        if (S.run && !*S.run) continue;
        const bool fresh = S.ghat != staged;
        if (fresh) {
            __syncthreads();  // the previous system's multiply has finished with the old slice
            const int nf = d.nz + 1;
            for (int i = threadIdx.x; i < nf * 6 * TX; i += blockDim.x) {
                const int lx = i % TX;
                const int r = i / TX;
                const int c = r % 6;
                const int fz = r / 6;
                const int kx = x0 + lx;
                if (kx < d.Lx) {
                    const int fx = kx <= d.nx ? kx : d.Lx - kx;
                    cp_async_elem(&sG[fz * GS + c * TX + lx],
                                  S.ghat + c * NO + ((long long)fz * (d.ny + 1) + fy) * (d.nx + 1) + fx);
                }
            }
            cp_async_commit();
            staged = S.ghat;
        }
        const C* __restrict__ src = pick<C>(S, src_sel) + (long long)cl * in_count * plane + col;
        C* __restrict__ dst = pick<C>(S, dst_sel) + (long long)cl * out_count * plane + col;
        auto ld_g = [&](int, int e) -> C {
            const int es = e - in_off;
            return (xin && es >= 0 && es < in_count) ? src[es * plane] : czero<C>();
        };
        auto st_s = [&](int l, int k, C v) { s[k * NL + l] = v; };
        fft4_io<A, B, -1, false, true, NL, A / 2 + 1, B>(s, tw, threadIdx.x, ld_g, st_s);
        if (fresh) {
            cp_async_wait_all();
            __syncthreads();
        }
        for (int i = threadIdx.x; i < L * TX; i += blockDim.x) {
            const int lx = i % TX;
            const int kz = i / TX;
            const int kx = x0 + lx;
            if (kx >= d.Lx) continue;
            const int fz = kz <= d.nz ? kz : L - kz;
            const unsigned mz = kz > d.nz ? SIGN_BIT : 0u;
            const unsigned mx = kx > d.nx ? SIGN_BIT : 0u;
            const C* g = sG + fz * GS + lx;
            // mirrored octant entries: the off-diagonal ij entry is odd in axes i and j
            const C G0 = g[0], G1 = g[TX], G2 = g[2 * TX];
            const C G3 = flip_sign(g[3 * TX], my ^ mz);
            const C G4 = flip_sign(g[4 * TX], mx ^ mz);
            const C G5 = flip_sign(g[5 * TX], mx ^ my);
            C* row = s + kz * NL + lx;
            const C q0 = row[0], q1 = row[TX], q2 = row[2 * TX];
            row[0] = gdot3<CONJ>(G0, q0, G5, q1, G4, q2);
            row[TX] = gdot3<CONJ>(G5, q0, G1, q1, G3, q2);
            row[2 * TX] = gdot3<CONJ>(G4, q0, G3, q1, G2, q2);
        }
        __syncthreads();
        auto ld_s = [&](int l, int e) -> C { return s[e * NL + l]; };
        auto st_g = [&](int, int k, C v) {
            const int eo = k - out_off;
            if (xin && eo >= 0 && eo < out_count) dst[eo * plane] = v;
        };
        fft4_io<A, B, 1, true, false, NL, A, B / 2 + 1>(s, tw, threadIdx.x, ld_s, st_g);
        __syncthreads();  // the next system's forward step writes s
    }
}

// Register-resident FP32 z pass for L = A * A, two y rows per block.  Block (x tile, j) serves the
// columns x0 .. x0 + TX - 1 of the rows ky = j and Ly - j (j = 0 and j = ny, their own mirror
// images, are served alone: the second half of the block repeats the first row's arithmetic and
// stores nothing).  Both rows read the same octant slice of the spectrum (fy = j; the odd entries
// flip sign in the mirrored row), so the slice is staged once for both and a warp's spectrum loads
// for the two rows are one shared-memory access.  Thread (lx, r, q) owns column x0 + lx of row r
// and, for each of the three components, the step-1 DFT of t = q and the step-2 DFT of k1 = q:
// the forward step 2 leaves X[q + A k2] (k2 = 0..A-1) of all three components in its registers,
// exactly the inputs of the inverse transform's step 1 for t = q, so the Green multiply runs in
// registers and each transform crosses shared memory once.  The nonzero inputs are loaded straight
// from global memory.  A block serves its columns for every system of the batch, restaging the
// spectrum slice only when the frequency changes.
template <bool CONJ, int A, int TX>
__global__ void __launch_bounds__(2 * TX * A, 3) k4z_pair(
    Dims d, const float2* __restrict__ tw, const ApplySys<float>* __restrict__ sys, int nsys, int in_count, int in_off,
    int out_count, int out_off, int src_sel, int dst_sel) {
    typedef float2 C;
    constexpr int L = A * A, NL = 2 * TX, NT = NL * A, NZ = A / 2 + 1;
    constexpr int E = 16;                                            // float2 per 128-byte bank row
    constexpr int YS = A * NL + (((NL - A * NL) % E) + E) % E;       // row stride of Y[t][.]
    const int nin = in_off + in_count;    // rows of a padded line that can be nonzero (<= NZ A)
    extern __shared__ unsigned char smem_raw[];
    C* sY = reinterpret_cast<C*>(smem_raw);   // two exchange buffers of A * YS, used alternately
    C* sG = sY + 2 * A * YS;              // [6][nz+1][TX] spectrum slice
    C* sW = sG + 6 * (d.nz + 1) * TX;     // twiddles exp(-2 pi i k / L), k < L
    const int lx = threadIdx.x % TX;
    const int r = (threadIdx.x / TX) & 1;
    const int q0 = threadIdx.x / NL;
    const int l = lx + TX * r;            // line of the exchange buffers
    const int j = blockIdx.y;             // 0 .. ny
    const bool alone = j == 0 || j == d.ny;
    const int ky = (r == 0 || alone) ? j : d.Ly - j;
    const bool owner = r == 0 || !alone;
    const int x0 = blockIdx.x * TX;
    const int kx = x0 + lx;
    const bool xin = kx < d.Lx;
    const unsigned my = ky > d.ny ? SIGN_BIT : 0u;
    const unsigned mx = kx > d.nx ? SIGN_BIT : 0u;
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const int GC = (d.nz + 1) * TX;
    const int plane = d.Ly * d.Lx;
    const long long colofs = (long long)ky * d.Lx + kx;
    for (int i = threadIdx.x; i < L; i += NT) sW[i] = tw[i];   // ordered before use by the first barrier
    const C* staged = nullptr;
    for (int si = 0; si < nsys; ++si) {
        // q re-read through an opaque move: everything derived from it (rows, offsets, masks,
        // twiddle indices) is recomputed per system instead of held in registers across systems
        int q;
        asm volatile("mov.u32 %0, %1;" : "=r"(q) : "r"(q0));
        const ApplySys<float> S = sys[si];
        if (S.run && !*S.run) continue;
        const bool fresh = S.ghat != staged;
        if (fresh) {
            __syncthreads();   // the previous slice's last reads (and the twiddle fill) are done
            // slice element i = (c (nz+1) + fz) TX + lxx; this thread copies i = tid + k NT
            const int lxx = threadIdx.x % TX;
            const int kxx = x0 + lxx;
            const int fx = kxx <= d.nx ? kxx : d.Lx - kxx;
            int row = threadIdx.x / TX;
            for (int i = threadIdx.x; i < 6 * GC; i += NT, row += NT / TX) {
                const int c = row / (d.nz + 1);
                const int fz = row - c * (d.nz + 1);
                if (kxx < d.Lx)
                    cp_async_elem(&sG[i], S.ghat + c * NO + ((long long)fz * (d.ny + 1) + j) * (d.nx + 1) + fx);
            }
            cp_async_commit();
            staged = S.ghat;
        }
        const C* __restrict__ src = pick<C>(S, src_sel) + colofs;
        C R[3][A];
        // ---- forward transforms, one component at a time through the exchange buffers
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C v[A];
            const C* xc = src + (long long)c * in_count * plane;
            // at most A/2 + 1 nonzero inputs per step-1 DFT (nin <= (A/2 + 1) A, checked at launch)
#pragma unroll
            for (int a = 0; a < A; ++a) {
                const int e = q + A * a;
                const int es = e - in_off;
                v[a] = (a < NZ && e < nin && es >= 0 && xin) ? xc[(long long)es * plane] : czero<C>();
            }
            dft_reg_p<A, -1, NZ, A>(v);
            if (q) {
#pragma unroll
                for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], lds_fresh(&sW[q * k1]));
            }
            // buffer c & 1 was last read two components ago, before the previous barrier
            C* Y = sY + (c & 1) * A * YS;
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) Y[q * YS + k1 * NL + l] = v[k1];
            __syncthreads();
#pragma unroll
            for (int t = 0; t < A; ++t) R[c][t] = Y[t * YS + q * NL + l];
            dft_reg<A, -1>(R[c]);   // R[c][k2] = X_c[q + A k2]
        }
        if (fresh) {
            cp_async_wait_all();
            __syncthreads();
        }
        // ---- Green multiply in registers
        if (xin) {
#pragma unroll
            for (int k2 = 0; k2 < A; ++k2) {
                const int kz = q + A * k2;
                const int fz = kz <= d.nz ? kz : L - kz;
                const unsigned mz = kz > d.nz ? SIGN_BIT : 0u;
                const C* g = sG + fz * TX + lx;
                const C G0 = g[0], G1 = g[GC], G2 = g[2 * GC];
                const C G3 = flip_sign(g[3 * GC], my ^ mz);
                const C G4 = flip_sign(g[4 * GC], mx ^ mz);
                const C G5 = flip_sign(g[5 * GC], mx ^ my);
                const C qa = R[0][k2], qb = R[1][k2], qc = R[2][k2];
                R[0][k2] = gdot3<CONJ>(G0, qa, G5, qb, G4, qc);
                R[1][k2] = gdot3<CONJ>(G5, qa, G1, qb, G3, qc);
                R[2][k2] = gdot3<CONJ>(G4, qa, G3, qb, G2, qc);
            }
        }
        // ---- inverse transforms: step 1 of t = q takes R[c][a] as its input a
        C* __restrict__ dst = pick<C>(S, dst_sel) + colofs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dft_reg<A, 1>(R[c]);
            if (q) {
#pragma unroll
                for (int k1 = 1; k1 < A; ++k1) R[c][k1] = cmulc(R[c][k1], lds_fresh(&sW[q * k1]));
            }
            // buffers continue the alternation: inverse c uses (c + 1) & 1, last read before the
            // barrier of the component before
            C* Y = sY + ((c + 1) & 1) * A * YS;
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) Y[q * YS + k1 * NL + l] = R[c][k1];
            __syncthreads();
            C v[A];
#pragma unroll
            for (int t = 0; t < A; ++t) v[t] = Y[t * YS + q * NL + l];
            dft_reg_p<A, 1, A, NZ>(v);   // outputs k < (A/2 + 1) A only (checked at launch)
            C* dc = dst + (long long)c * out_count * plane;
#pragma unroll
            for (int k2 = 0; k2 < NZ; ++k2) {
                const int eo = q + A * k2 - out_off;
                if (owner && xin && eo >= 0 && eo < out_count) dc[(long long)eo * plane] = v[k2];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// z pass with the Green multiply: forward z FFT, u-hat = G-hat q-hat (conj G-hat for the
// adjoint), inverse z FFT.  CTA: TX lines along x at one ky, all three components.
// src [3][in_count][Ly][Lx] (sel), dst [3][out_count][Ly][Lx] (sel)
// ---------------------------------------------------------------------------------------------
template <typename T, bool CONJ, class F>
__global__ void LSM_FFT_BOUND(T, F) k_fftz_green(Dims d, FftPlan pz, const typename cplx_of<T>::type* __restrict__ tw,
                                                    const ApplySys<T>* __restrict__ sys, int TX, int in_count, int in_off,
                                                    int out_count, int out_off, int src_sel, int dst_sel) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    const ApplySys<T> S = sys[blockIdx.z];
    if (S.run && !*S.run) return;
    const int L = d.Lz, NL = 3 * TX;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = F::INPLACE ? sa : sa + (size_t)L * NL;
    const int ky = blockIdx.y;
    const int x0 = blockIdx.x * TX;
    const long long plane = (long long)d.Ly * d.Lx;
    const C* src = pick<C>(S, src_sel);
    C* dst = pick<C>(S, dst_sel);
    const long long s_c = (long long)in_count * plane, d_c = (long long)out_count * plane;
    for (int i = threadIdx.x; i < L * NL; i += blockDim.x) {
        const int lx = i % TX;
        const int rest = i / TX;
        const int c = rest % 3;
        const int e = rest / 3;
        const int x = x0 + lx;
        const int es = e - in_off;
        C v = czero<C>();
        if (x < d.Lx && es >= 0 && es < in_count) v = src[c * s_c + es * plane + (long long)ky * d.Lx + x];
        sa[e * NL + c * TX + lx] = v;
    }
    __syncthreads();
    C* r = F::template run<-1>(sa, sb, pz, NL, NL, tw);
    C* o = (r == sa) ? sb : sa;
    for (int i = threadIdx.x; i < L * TX; i += blockDim.x) {
        const int lx = i % TX;
        const int kz = i / TX;
        const int kx = x0 + lx;
        if (kx >= d.Lx) continue;
        C G[6];
        ghat_at(S.ghat, d, kx, ky, kz, CONJ, G);
        C* row = r + kz * NL + lx;
        const C q0 = row[0], q1 = row[TX], q2 = row[2 * TX];
        row[0] = cadd(cadd(cmul(G[0], q0), cmul(G[5], q1)), cmul(G[4], q2));
        row[TX] = cadd(cadd(cmul(G[5], q0), cmul(G[1], q1)), cmul(G[3], q2));
        row[2 * TX] = cadd(cadd(cmul(G[4], q0), cmul(G[3], q1)), cmul(G[2], q2));
    }
    __syncthreads();
    C* r2 = F::template run<1>(r, o, pz, NL, NL, tw);
    for (int i = threadIdx.x; i < out_count * NL; i += blockDim.x) {
        const int lx = i % TX;
        const int rest = i / TX;
        const int c = rest % 3;
        const int eo = rest / 3;
        const int x = x0 + lx;
        if (x < d.Lx) dst[c * d_c + eo * plane + (long long)ky * d.Lx + x] = r2[(eo + out_off) * NL + c * TX + lx];
    }
}

// ---------------------------------------------------------------------------------------------
// inverse FFT along x + crop + Au = u - u_s.  CTA: B rows y at one z, 3 comps.  src w1 [3][nz][ny][Lx]
// ---------------------------------------------------------------------------------------------
template <typename T, class F>
__global__ void LSM_FFT_BOUND(T, F) k_fftx_out(Dims d, const ApplySys<T>* __restrict__ sys, FftPlan px,
                                                  const typename cplx_of<T>::type* __restrict__ tw, int B, int xoff) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    const ApplySys<T> S = sys[blockIdx.z];
    if (S.run && !*S.run) return;
    const int NL = 3 * B, LD = NL + 1, L = d.Lx;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = F::INPLACE ? sa : sa + (size_t)L * LD;
    const int z = blockIdx.y;
    const int y0 = blockIdx.x * B;
    const C* __restrict__ src = S.w2;
    for (int i = threadIdx.x; i < NL * L; i += blockDim.x) {
        const int kx = i % L;
        const int l = i / L;
        const int c = l / B;
        const int y = y0 + (l % B);
        C v = czero<C>();
        if (y < d.ny) v = src[(((long long)c * d.nz + z) * d.ny + y) * L + kx];
        sa[kx * LD + l] = v;
    }
    __syncthreads();
    C* r = F::template run<1>(sa, sb, px, NL, LD, tw);
    for (int i = threadIdx.x; i < NL * d.nx; i += blockDim.x) {
        const int x = i % d.nx;
        const int l = i / d.nx;
        const int c = l / B;
        const int y = y0 + (l % B);
        if (y < d.ny) {
            const long long idx = (((long long)c * d.nz + z) * d.ny + y) * d.nx + x;
            S.out[idx] = csub(S.u[idx], r[(x + xoff) * LD + l]);
        }
    }
    if (S.count && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(S.count, 1ull);
}

// ---------------------------------------------------------------------------------------------
// contrast source on the extended nodes: q_j = sum_k D_k sigma_jk + w^2 drho u_j, q [3][ez][ey][ex]
// (index p holds node p - 1).  sigma in w1, q written to w2.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 ? 6 : 1) k_divq(Dims d, const T* __restrict__ drho, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const C* __restrict__ sig = S.w1;
    const C* __restrict__ u = S.u;
    C* __restrict__ q = S.w2;
    const long long N = d.N;
    const long long E = (long long)d.ex * d.ey * d.ez;
    const long long sxy = (long long)d.nx * d.ny;
    const T i2h = (T)(0.5 / d.h);
    for (long long idx = (long long)blockIdx.x * NTH + threadIdx.x; idx < E; idx += (long long)gridDim.x * NTH) {
        const int p0 = (int)(idx % d.ex) - 1;
        const int p1 = (int)((idx / d.ex) % d.ey) - 1;
        const int p2 = (int)(idx / ((long long)d.ex * d.ey)) - 1;
        const int p[3] = {p0, p1, p2};
        const int nn[3] = {d.nx, d.ny, d.nz};
        const long long st[3] = {1, (long long)d.nx, sxy};
        const bool in0 = p0 >= 0 && p0 < d.nx, in1 = p1 >= 0 && p1 < d.ny, in2 = p2 >= 0 && p2 < d.nz;
        const long long base = (long long)p2 * sxy + (long long)p1 * d.nx + p0;
        C qj[3] = {czero<C>(), czero<C>(), czero<C>()};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // the neighbours p +- e_k are model nodes when the other two coordinates are inside
            // and p_k + 1 (resp. p_k - 1) is inside along k; loads are predicated, not branched
            const bool other = (k == 0 ? (in1 && in2) : (k == 1 ? (in0 && in2) : (in0 && in1)));
            const bool hi = other && p[k] + 1 >= 0 && p[k] + 1 < nn[k];
            const bool lo = other && p[k] - 1 >= 0 && p[k] - 1 < nn[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const C* sJ = sig + (long long)t2v(j, k) * N + base;
                const C vh = hi ? sJ[st[k]] : czero<C>();
                const C vl = lo ? sJ[-st[k]] : czero<C>();
                qj[j] = cadd(qj[j], csub(vh, vl));
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) qj[j] = cscale(qj[j], i2h);
        if (in0 && in1 && in2) {
            const T w = S.omega2 * __ldg(&drho[base]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const C uj = u[j * N + base];
                qj[j].x += w * uj.x;
                qj[j].y += w * uj.y;
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) q[j * E + idx] = qj[j];
    }
}

// four-step contiguous-rows FFT: NL rows per block, compile-time sizes, loads batched in registers.
// Row r of src starts at src + r * in_count (placed at in_off), row r of dst at dst + r * out_count.
template <typename T, int DIR, int A, int B, int NL>
__global__ void __launch_bounds__(NL * FourStep<A LSM_COMMA B>::TPL, sizeof(T) == 8 ? 3 : 2) k4_rows(const typename cplx_of<T>::type* __restrict__ tw,
                                                                  const ApplySys<T>* __restrict__ sys, int src_sel, int dst_sel,
                                                                  long long nrows, int in_count, int in_off, int out_count,
                                                                  int out_off) {
    typedef typename cplx_of<T>::type C;
    constexpr int L = A * B, TPL = FourStep<A, B>::TPL, NTHR = NL * TPL, LD = NL + 1, PER = L / TPL;
    extern __shared__ unsigned char smem_raw[];
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    C* s = reinterpret_cast<C*>(smem_raw);
    const C* __restrict__ src = pick<C>(S, src_sel);
    C* __restrict__ dst = pick<C>(S, dst_sel);
    const long long r0 = (long long)blockIdx.x * NL;
    const int tid = threadIdx.x;
    C v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHR;
        const int e = i % L, l = i / L;
        const long long row = r0 + l;
        const int es = e - in_off;
        v[k] = (row < nrows && es >= 0 && es < in_count) ? src[row * in_count + es] : czero<C>();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHR;
        s[(i % L) * LD + i / L] = v[k];
    }
    __syncthreads();
    fft4_smem<A, B, DIR, (DIR < 0 ? A / 2 + 1 : A), (DIR > 0 ? B / 2 + 1 : B)>(s, NL, LD, tw, tid);   // as in k4_strided
    for (int i = tid; i < NL * out_count; i += NTHR) {
        const int e = i % out_count, l = i / out_count;
        const long long row = r0 + l;
        if (row < nrows) dst[row * out_count + e] = s[(e + out_off) * LD + l];
    }
}

// Two-step FFT of contiguous rows for L = A * A with each line held by A consecutive lanes of one
// warp: lane q owns the step-1 DFT of t = q and the step-2 DFT of k1 = q.  Step 1 loads its inputs
// x[t + A a] straight from global memory (for each a the line's lanes read A consecutive
// elements), the transpose between the steps goes through a shared-memory tile private to the
// line (row stride A + 1: conflict-free both ways) ordered by __syncwarp, and step 2 leaves
// X[k1 + A k2] in registers for a coalesced store.  No block barrier and one shared-memory round
// trip per element (the tile-transposing kernels above make three).  The arithmetic is that of
// fft4_smem, operation for operation, so results are bitwise those of k4_rows / k4_fftx_out.
template <int A, typename C>
__device__ __forceinline__ void rows_w_exchange(C (&v)[A], C* tl, int q) {
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) tl[q * (A + 1) + k1] = v[k1];
    __syncwarp();
#pragma unroll
    for (int t = 0; t < A; ++t) v[t] = tl[t * (A + 1) + q];
}

// forward x FFT of zero-padded rows: row r of src (in_count elements, the rest zero, at most
// (A/2 + 1) A of them) -> row r of dst (L elements)
template <typename T, int A, int LPB>
__global__ void __launch_bounds__(LPB * A, sizeof(T) == 4 ? 4 : 1) k4_rows_w(const typename cplx_of<T>::type* __restrict__ tw,
                                                     const ApplySys<T>* __restrict__ sys, int src_sel, int dst_sel,
                                                     long long nrows, int in_count) {
    typedef typename cplx_of<T>::type C;
    constexpr int L = A * A;
    __shared__ C tile[LPB][A * (A + 1)];
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const int ln = threadIdx.x / A, q = threadIdx.x % A;
    const long long row = (long long)blockIdx.x * LPB + ln;
    const bool live = row < nrows;
    const C* __restrict__ src = pick<C>(S, src_sel) + row * in_count;
    C* __restrict__ dst = pick<C>(S, dst_sel) + row * L;
    C v[A];
#pragma unroll
    for (int a = 0; a < A; ++a) {
        const int e = q + A * a;
        v[a] = (a < A / 2 + 1 && live && e < in_count) ? src[e] : czero<C>();
    }
    dft_reg_p<A, -1, A / 2 + 1, A>(v);
    if (q) {
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], __ldg(&tw[q * k1]));
    }
    rows_w_exchange<A>(v, tile[ln], q);
    dft_reg_p<A, -1, A, A>(v);
    if (live) {
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) dst[q + A * k2] = v[k2];
    }
}

// blocks per SM each precision is compiled for: FP32 (with or without DOTS) fits 80 registers
// for 3 blocks of 256 threads; FP64 and double-float keep the occupancy they reach unconstrained
// (5 and 4 blocks of 128 threads at A = 16)
template <typename T>
constexpr int xout_min_blocks() { return sizeof(T) == 4 ? 3 : (std::is_same<T, dfloat>::value ? 4 : 5); }

// inverse x FFT of the rows of w2 [3][nz][ny][L], crop to x = k - xoff in [0, nx) (at most
// (A/2 + 1) A outputs), Au = u - u_s.
// DOTS (FP32 only): each warp also writes to the system's DotSink its partial sums of the BiCGSTAB
// inner product that needs this output, and dot_finish adds the warps' partials in FP64 and
// finishes alpha or omega.  DOT_RV: <r^, Au>; r^ at the thread's outputs is copied to shared
// memory (cp.async, dynamic shared memory [LPB][NO][A]) while the transform runs.  DOT_TS: <Au, u>
// and <Au, Au>, from registers.  Within a warp the sums are plain FP32: at most 2 (A/2 + 1)
// products per thread and sum and a 5-level shuffle tree, so within about (A + 7) 2^-24 of the
// exact sum relative to the sum of |products| (1.4e-6 at A = 16): the accuracy of an FP32
// BiCGSTAB's own inner products, where the apply itself carries FP32 rounding.  (Compensated sums
// as in the vector kernels doubled this kernel's instructions and registers; a block reduction
// and a last-block ticket stalled every block on a barrier or an atomic round trip.)
template <typename T, int A, int LPB, int DOTS = 0>
__global__ void __launch_bounds__(LPB * A, xout_min_blocks<T>()) k4_xout_w(Dims d, const ApplySys<T>* __restrict__ sys,
                                                     const typename cplx_of<T>::type* __restrict__ tw, int xoff) {
    typedef typename cplx_of<T>::type C;
    constexpr int L = A * A, NO = A / 2 + 1;
    static_assert(DOTS == 0 || sizeof(T) == 4, "inner products are folded into the FP32 epilogue only");
    __shared__ C tile[LPB][A * (A + 1)];
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const int ln = threadIdx.x / A, q = threadIdx.x % A;
    const long long nrows = 3LL * d.nz * d.ny;
    const long long row = (long long)blockIdx.x * LPB + ln;
    const bool live = row < nrows;
    const C* __restrict__ src = S.w2 + row * L;
    const C* __restrict__ uin = S.u + row * d.nx;
    C* __restrict__ out = S.out + row * d.nx;
    const DotSink* D = nullptr;
    C* rhs = nullptr;   // DOT_RV: this thread's r^ values, [k2] at stride A
    if constexpr (DOTS == DOT_RV) {
        extern __shared__ __align__(16) unsigned char rh_smem[];
        D = static_cast<const DotSink*>(S.dot);
        rhs = reinterpret_cast<C*>(rh_smem) + ln * NO * A + q;
        const C* __restrict__ rh = static_cast<const C*>(D->rh) + row * d.nx;
        if (live) {
#pragma unroll
            for (int k2 = 0; k2 < NO; ++k2) {
                const int x = q + A * k2 - xoff;
                if (x >= 0 && x < d.nx) cp_async_elem(&rhs[k2 * A], &rh[x]);
            }
        }
        cp_async_commit();
    } else if constexpr (DOTS == DOT_TS) {
        D = static_cast<const DotSink*>(S.dot);
    }
    C v[A];
#pragma unroll
    for (int a = 0; a < A; ++a) v[a] = live ? src[q + A * a] : czero<C>();
    // FP32: u for the epilogue is fetched now, so its latency overlaps the transform
    constexpr bool PRE = sizeof(T) == 4;
    C uo[PRE ? NO : 1];
    if constexpr (PRE) {
#pragma unroll
        for (int k2 = 0; k2 < NO; ++k2) {
            const int x = q + A * k2 - xoff;
            uo[k2] = (live && x >= 0 && x < d.nx) ? uin[x] : czero<C>();
        }
    }
    dft_reg_p<A, 1, A, A>(v);
    if (q) {
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) {
            C w = __ldg(&tw[q * k1]);
            w.y = -w.y;
            v[k1] = cmul(v[k1], w);
        }
    }
    rows_w_exchange<A>(v, tile[ln], q);
    dft_reg_p<A, 1, A, NO>(v);
    if constexpr (DOTS != 0) {
        if constexpr (DOTS == DOT_RV) cp_async_wait_all();   // own copies only: no barrier
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;   // Re, Im of the inner product; |Au|^2
        if (live) {
#pragma unroll
            for (int k2 = 0; k2 < NO; ++k2) {
                const int x = q + A * k2 - xoff;
                if (x >= 0 && x < d.nx) {
                    const C u = uo[PRE ? k2 : 0];
                    const C o = csub(u, v[k2]);
                    out[x] = o;
                    // conj(a) b with a = r^, b = Au (alpha) or a = Au, b = u (omega)
                    if constexpr (DOTS == DOT_RV) {
                        const C a = rhs[k2 * A];
                        s0 = fmaf(a.x, o.x, fmaf(a.y, o.y, s0));
                        s1 = fmaf(a.x, o.y, fmaf(-a.y, o.x, s1));
                    } else {
                        s0 = fmaf(o.x, u.x, fmaf(o.y, u.y, s0));
                        s1 = fmaf(o.x, u.y, fmaf(-o.y, u.x, s1));
                        s2 = fmaf(o.x, o.x, fmaf(o.y, o.y, s2));
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            if constexpr (DOTS == DOT_TS) s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            const long long part = (long long)blockIdx.x * (LPB * A / 32) + (threadIdx.x >> 5);
            reinterpret_cast<float4*>(D->partials)[part] = make_float4(s0, s1, s2, 0.f);
        }
    } else if (live) {
#pragma unroll
        for (int k2 = 0; k2 < NO; ++k2) {
            const int x = q + A * k2 - xoff;
            if (x >= 0 && x < d.nx) out[x] = csub(PRE ? uo[PRE ? k2 : 0] : uin[x], v[k2]);
        }
    }
    if (S.count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.count, 1ull);
}

// four-step inverse x FFT + crop + Au = u - u_s; ROWS rows x 3 components per block; src w2.
template <typename T, int A, int B, int ROWS>
__global__ void __launch_bounds__(3 * ROWS * FourStep<A LSM_COMMA B>::TPL, sizeof(T) == 8 ? 3 : 2) k4_fftx_out(Dims d, const ApplySys<T>* __restrict__ sys,
                                                                      const typename cplx_of<T>::type* __restrict__ tw,
                                                                      int xoff) {
    typedef typename cplx_of<T>::type C;
    constexpr int L = A * B, TPL = FourStep<A, B>::TPL, NL = 3 * ROWS, NTHR = NL * TPL, LD = NL + 1, PER = L / TPL;
    extern __shared__ unsigned char smem_raw[];
    const ApplySys<T> S = sys[blockIdx.z];
    if (S.run && !*S.run) return;
    C* s = reinterpret_cast<C*>(smem_raw);
    const int z = blockIdx.y;
    const int y0 = blockIdx.x * ROWS;
    const C* __restrict__ src = S.w2;
    const int tid = threadIdx.x;
    C v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHR;
        const int kx = i % L, l = i / L;
        const int c = l / ROWS, y = y0 + l % ROWS;
        v[k] = (y < d.ny) ? src[(((long long)c * d.nz + z) * d.ny + y) * L + kx] : czero<C>();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHR;
        s[(i % L) * LD + i / L] = v[k];
    }
    // FP32: u for the epilogue is fetched now, so its latency overlaps the transform (nx = L / 2);
    // FP64 is bound by its arithmetic, and the registers cost it occupancy, so it reads u at the end
    constexpr int NX = L / 2, PO = NL * NX / NTHR;
    constexpr bool PRE = sizeof(T) == 4;
    const C* __restrict__ uin = S.u;
    C uo[PRE ? PO : 1];
    if constexpr (PRE) {
#pragma unroll
        for (int k = 0; k < PO; ++k) {
            const int i = tid + k * NTHR;
            const int x = i % NX, l = i / NX;
            const int c = l / ROWS, y = y0 + l % ROWS;
            uo[k] = (y < d.ny) ? uin[(((long long)c * d.nz + z) * d.ny + y) * NX + x] : czero<C>();
        }
    }
    __syncthreads();
    fft4_smem<A, B, 1, A, B / 2 + 1>(s, NL, LD, tw, tid);   // outputs x + xoff <= L/2 only
    C* __restrict__ out = S.out;
#pragma unroll
    for (int k = 0; k < PO; ++k) {
        const int i = tid + k * NTHR;
        const int x = i % NX, l = i / NX;
        const int c = l / ROWS, y = y0 + l % ROWS;
        if (y < d.ny) {
            const long long idx = (((long long)c * d.nz + z) * d.ny + y) * NX + x;
            const C uv = PRE ? uo[PRE ? k : 0] : uin[idx];
            out[idx] = csub(uv, s[(x + xoff) * LD + l]);
        }
    }
    if (S.count && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(S.count, 1ull);
}

// ---------------------------------------------------------------------------------------------
// generic contiguous-rows pass: NL rows per CTA.  Row r of src starts at src + r*in_count (elements
// placed at in_off), row r of dst at dst + r*out_count (elements read from out_off).
// ---------------------------------------------------------------------------------------------
template <int DIR, typename C>
__device__ __forceinline__ void rows_tile(const C* src, C* dst, const FftPlan& p, const C* __restrict__ tw,
                                          long long r0, long long nrows, int NL, int in_count, int in_off,
                                          int out_count, int out_off, C* sa, C* sb) {
    const int L = p.L, LD = NL + 1;
    for (int i = threadIdx.x; i < NL * L; i += NTH) {
        const int e = i % L;
        const int l = i / L;
        const long long row = r0 + l;
        const int es = e - in_off;
        C v = czero<C>();
        if (row < nrows && es >= 0 && es < in_count) v = src[row * in_count + es];
        sa[e * LD + l] = v;
    }
    __syncthreads();
    C* r = fft_smem<DIR>(sa, sb, p, NL, LD, tw, threadIdx.x, NTH);
    for (int i = threadIdx.x; i < NL * out_count; i += NTH) {
        const int e = i % out_count;
        const int l = i / out_count;
        const long long row = r0 + l;
        if (row < nrows) dst[row * out_count + e] = r[(e + out_off) * LD + l];
    }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(NTH) k_rows(FftPlan p, const typename cplx_of<T>::type* __restrict__ tw,
                                              const ApplySys<T>* __restrict__ sys, int src_sel, int dst_sel,
                                              long long nrows, int NL, int in_count, int in_off, int out_count, int out_off) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = sa + (size_t)p.L * (NL + 1);
    rows_tile<DIR>(pick<C>(S, src_sel), pick<C>(S, dst_sel), p, tw, (long long)blockIdx.x * NL, nrows, NL,
                   in_count, in_off, out_count, out_off, sa, sb);
}

template <typename T, int DIR>
__global__ void __launch_bounds__(NTH) k_rows_raw(FftPlan p, const typename cplx_of<T>::type* __restrict__ tw,
                                                  const typename cplx_of<T>::type* src, typename cplx_of<T>::type* dst,
                                                  long long nrows, int NL) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ unsigned char smem_raw[];
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = sa + (size_t)p.L * (NL + 1);
    rows_tile<DIR>(src, dst, p, tw, (long long)blockIdx.x * NL, nrows, NL, p.L, 0, p.L, 0, sa, sb);
}

// ---------------------------------------------------------------------------------------------
// adjoint: transposed divergence and contraction.  z (extended nodes) in w1 [3][ez][ey][ex];
// writes c_K = sum_J dC_JK tau_J into w2 [6][N], tau_J = sum_{(j,k)->J} D_k^T z_j.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTH) k_adj_stress(Dims d, const T* __restrict__ dC, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const C* __restrict__ z = S.w1;
    C* __restrict__ cc = S.w2;
    const long long N = d.N;
    const long long E = (long long)d.ex * d.ey * d.ez;
    const T i2h = (T)(0.5 / d.h);
    const long long sxy = (long long)d.nx * d.ny;
    for (long long idx = (long long)blockIdx.x * NTH + threadIdx.x; idx < N; idx += (long long)gridDim.x * NTH) {
        const int ix = (int)(idx % d.nx);
        const int iy = (int)((idx / d.nx) % d.ny);
        const int iz = (int)(idx / sxy);
        // extended index of node (ix, iy, iz) is (ix+1, iy+1, iz+1)
        const long long e0 = ((long long)(iz + 1) * d.ey + (iy + 1)) * d.ex + (ix + 1);
        const long long st[3] = {1, (long long)d.ex, (long long)d.ex * d.ey};
        C tau[6];
#pragma unroll
        for (int J = 0; J < 6; ++J) tau[J] = czero<C>();
#pragma unroll
        for (int j = 0; j < 3; ++j) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const C* zj = z + j * E;
                const C v = csub(zj[e0 - st[k]], zj[e0 + st[k]]);
                const int J = t2v(j, k);
                tau[J] = cadd(tau[J], v);
            }
        }
        T c21[21];
#pragma unroll
        for (int k = 0; k < 21; ++k) c21[k] = __ldg(&dC[k * N + idx]);
#pragma unroll
        for (int K = 0; K < 6; ++K) {
            C s = czero<C>();
#pragma unroll
            for (int J = 0; J < 6; ++J) {
                const T c = c21[p21(J, K)];
                s.x += c * tau[J].x;
                s.y += c * tau[J].y;
            }
            cc[K * N + idx] = cscale(s, i2h);
        }
    }
}

// transpose of the Eq. 18 derivative along one axis, at node i of n, for field f with stride s
template <typename C, typename T>
__device__ __forceinline__ C dT_axis(const C* f, long long idx, int i, int n, long long s, T ih, T i2h) {
    C acc = czero<C>();
    // interior rows i-1 and i+1 (rows 1..n-2 use the central difference)
    if (i - 1 >= 1 && i - 1 <= n - 2) acc = cadd(acc, cscale(f[idx - s], i2h));
    if (i + 1 >= 1 && i + 1 <= n - 2) acc = csub(acc, cscale(f[idx + s], i2h));
    // boundary row 0: (f1 - f0)/h
    if (i == 0) acc = csub(acc, cscale(f[idx], ih));
    if (i == 1) acc = cadd(acc, cscale(f[idx - s], ih));
    // boundary row n-1: (f_{n-1} - f_{n-2})/h
    if (i == n - 2) acc = csub(acc, cscale(f[idx + s], ih));
    if (i == n - 1) acc = cadd(acc, cscale(f[idx], ih));
    return acc;
}

// AH w = w - (E^T c + w^2 drho z)
template <typename T>
__global__ void __launch_bounds__(NTH) k_adj_out(Dims d, const T* __restrict__ drho, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const C* __restrict__ cc = S.w2;
    const C* __restrict__ z = S.w1;
    const long long N = d.N;
    const long long E = (long long)d.ex * d.ey * d.ez;
    const T ih = (T)(1.0 / d.h), i2h = (T)(0.5 / d.h);
    const long long sxy = (long long)d.nx * d.ny;
    for (long long idx = (long long)blockIdx.x * NTH + threadIdx.x; idx < N; idx += (long long)gridDim.x * NTH) {
        const int ix = (int)(idx % d.nx);
        const int iy = (int)((idx / d.nx) % d.ny);
        const int iz = (int)(idx / sxy);
        const int ii[3] = {ix, iy, iz};
        const int nn[3] = {d.nx, d.ny, d.nz};
        const long long ss[3] = {1, (long long)d.nx, sxy};
        const long long e0 = ((long long)(iz + 1) * d.ey + (iy + 1)) * d.ex + (ix + 1);
        const T w = S.omega2 * __ldg(&drho[idx]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            C acc = czero<C>();
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc = cadd(acc, dT_axis(cc + (long long)t2v(i, a) * N, idx, ii[a], nn[a], ss[a], ih, i2h));
            const C zi = z[i * E + e0];
            acc.x += w * zi.x;
            acc.y += w * zi.y;
            S.out[i * N + idx] = csub(S.u[i * N + idx], acc);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------
#ifndef LSM_APPLY_DFLOAT_TU
void apply_ws_elems(const Dims& d, int kernel, long long* w1, long long* w2) {
    if (kernel == 1) {
        // sampled-H form: w1 holds [9][N], then [9][nz][Ly][Lx], then [3][nz][Ly][Lx];
        // w2 holds [9][nz][ny][Lx], then the full transforms [9][Lz][Ly][Lx], then [3][nz][ny][Lx]
        const long long a = 9LL * d.nz * d.Ly * d.Lx;
        *w1 = a > 9 * d.N ? a : 9 * d.N;
        *w2 = 9LL * d.Lz * d.Ly * d.Lx;
        return;
    }
    // both buffers hold any intermediate of the apply or the adjoint
    const long long c[] = {
        6 * d.N,                           // sigma
        3LL * d.ex * d.ey * d.ez,          // q / z on the extended nodes
        3LL * d.ez * d.ey * d.Lx,          // after the x FFT
        3LL * d.ez * d.Ly * d.Lx,          // after the y FFT
        3LL * d.nz * d.Ly * d.Lx,          // after the z pass
        3LL * d.nz * d.ny * d.Lx,          // after the inverse y FFT / first adjoint pass
    };
    long long m = 0;
    for (long long v : c) m = v > m ? v : m;
    *w1 = m;
    *w2 = m;
}
#endif

static const size_t SMEM_CAP = 96 * 1024;

template <typename T>
static int rows_per_tile(int L) {
    typedef typename cplx_of<T>::type C;
    // 3 comps x B rows, ping-pong, padded leading dimension
    int B = 8;
    while (B > 1 && 2 * (size_t)L * (3 * B + 1) * sizeof(C) > SMEM_CAP) --B;
    return B;
}
// Tiles of the generic engine; shrink halves them (a schedule variant, see Schedule).
template <typename T>
static int strided_tx(int L, int ncomp, int shrink = 0) {
    typedef typename cplx_of<T>::type C;
    int TX = sizeof(T) == 4 ? 16 : 8;
    while (TX > 1 && 2 * (size_t)L * ncomp * TX * sizeof(C) > SMEM_CAP) TX /= 2;
    TX >>= shrink;
    return TX > 1 ? TX : 1;
}
template <typename T>
static int generic_rows_nl(int L, int shrink = 0) {
    typedef typename cplx_of<T>::type C;
    int NL = 16;
    while (NL > 1 && 2 * (size_t)L * (NL + 1) * sizeof(C) > SMEM_CAP) NL /= 2;
    NL >>= shrink;
    return NL > 1 ? NL : 1;
}

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

static inline int grid_elems(long long n) {
    long long b = (n + NTH - 1) / NTH;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

// First use of a kernel: raise its dynamic shared-memory limit whenever a launch needs more than
// 48 KB.  The L1 / shared-memory split is left to the driver, which sizes it for the kernel's
// resident blocks: forcing the largest shared carveout left 28 KB of L1 and slowed the FP32 z
// pass from 201 to 235 us per system apply (its spills and cached loads missed L1) and the FP32
// inverse y pass from 46 to 57 us.
// static_sm: the kernel's static shared memory; the dynamic limit must be raised once
// static + dynamic passes 48 KB
static void smem_attr(const void* k, size_t sm, size_t static_sm = 0) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> seen;
    std::lock_guard<std::mutex> lk(mu);
    const bool big = sm + static_sm > 48 * 1024;
    for (auto& e : seen)
        if (e.first == k) {
            if (e.second >= sm) return;
            if (big) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            e.second = sm;
            return;
        }
    if (big) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    seen.push_back({k, sm});
}

// The two-step kernels prune at compile time: a line of length L = A B has at most A/2 + 1
// nonzero inputs per step-1 DFT and at most B/2 + 1 wanted outputs per step-2 DFT.  True when a
// line with nonzero inputs below in_end and wanted outputs below out_end fits that; the
// padded lines here (at most n + 2 = L/2 + 2 of either) always do.
static bool fourstep_prunable(int L, int in_end, int out_end) {
    int A, B;
    switch (L) {
        case 16: A = 4; B = 4; break;
        case 32: A = 4; B = 8; break;
        case 64: A = 8; B = 8; break;
        case 128: A = 8; B = 16; break;
        case 256: A = 16; B = 16; break;
        case 512: A = 16; B = 32; break;
        default: return true;   // generic engine
    }
    return in_end <= (A / 2 + 1) * B && out_end <= A * (B / 2 + 1);
}

// Call fn with the FFT engine for line length L: compile-time four-step for 16..512 unless the
// schedule variant v asks for the generic engine (v = 1, 2), else generic.
// ONLY256 (the double-float operator): the compile-time engine for L = 256 only, every other length
// generic, which keeps that translation unit's build short.
template <bool ONLY256 = false, typename Fn>
static void with_engine(int L, Fn&& fn, int v = 0) {
    if constexpr (ONLY256) {
        if (L == 256 && v != 1 && v != 2) fn(FourStepFFT<16, 16>());
        else fn(GenericFFT());
    } else {
        if (v == 1 || v == 2) {
            fn(GenericFFT());
            return;
        }
        switch (L) {
            case 16: fn(FourStepFFT<4, 4>()); break;
            case 32: fn(FourStepFFT<4, 8>()); break;
            case 64: fn(FourStepFFT<8, 8>()); break;
            case 128: fn(FourStepFFT<8, 16>()); break;
            case 256: fn(FourStepFFT<16, 16>()); break;
            case 512: fn(FourStepFFT<16, 32>()); break;
            default: fn(GenericFFT()); break;
        }
    }
}

// tile of B rows x 3 components for the contiguous x passes
template <typename T, class F>
static void rows_cfg(int L, int& B, int& threads, size_t& sm, int shrink = 0) {
    typedef typename cplx_of<T>::type C;
    if constexpr (F::INPLACE) {
        B = sizeof(T) == 4 ? 8 : 4;
        threads = 3 * B * F::TPL;
        sm = (size_t)L * (3 * B + 1) * sizeof(C);
    } else {
        B = rows_per_tile<T>(L) >> shrink;
        if (B < 1) B = 1;
        threads = NTH;
        sm = 2 * (size_t)L * (3 * B + 1) * sizeof(C);
    }
}
// tile of TX consecutive lines x ncomp components for the strided passes
template <typename T, class F>
static void strided_cfg(int L, int ncomp, int& TX, int& threads, size_t& sm, int shrink = 0) {
    typedef typename cplx_of<T>::type C;
    if constexpr (F::INPLACE) {
        TX = sizeof(T) == 4 ? (ncomp == 1 ? 16 : 4) : (ncomp == 1 ? 8 : 4);
        threads = ncomp * TX * F::TPL;
        const size_t ybuf = (size_t)F::B_ * fft4_ystride<F::A_, C>(ncomp * TX);
        sm = (ybuf > (size_t)L * ncomp * TX ? ybuf : (size_t)L * ncomp * TX) * sizeof(C);
    } else {
        TX = strided_tx<T>(L, ncomp, shrink);
        threads = NTH;
        sm = 2 * (size_t)L * ncomp * TX * sizeof(C);
    }
}

// forward x FFT of the contrast source rows: w2 [3][ez][ey][ex] -> w1 [3][ez][ey][Lx]
template <typename T>
static void launch_xfwd(const Dims& d, const ApplySys<T>* sys, int nsys, const Plans& pl, cudaStream_t st, int v = 0) {
    typedef typename cplx_of<T>::type C;
    if (!fourstep_prunable(d.Lx, d.ex, 0)) v = 1;
    const long long nrows = 3LL * d.ez * d.ey;
    with_engine<std::is_same<T, dfloat>::value>(d.Lx, [&](auto eng) {
        using F = decltype(eng);
        if constexpr (F::INPLACE && F::A_ == F::B_) {
            constexpr int A = F::A_, LPB = sizeof(T) == 4 ? 16 : 8;
            k4_rows_w<T, A, LPB><<<dim3(cdiv(nrows, LPB), nsys), LPB * A, 0, st>>>((const C*)pl.twx, sys, 3, 2, nrows,
                                                                                   d.ex);
        } else if constexpr (F::INPLACE) {
            constexpr int A = F::A_, B = F::B_, NL = sizeof(T) == 4 ? 8 : 12;
            const size_t sm = (size_t)A * B * (NL + 1) * sizeof(C);
            smem_attr((const void*)k4_rows<T, -1, A, B, NL>, sm);
            k4_rows<T, -1, A, B, NL><<<dim3(cdiv(nrows, NL), nsys), NL * F::TPL, sm, st>>>(
                (const C*)pl.twx, sys, 3, 2, nrows, d.ex, 0, d.Lx, 0);
        } else {
            const int NL = generic_rows_nl<T>(d.Lx, v == 2);
            const size_t sm = 2 * (size_t)d.Lx * (NL + 1) * sizeof(C);
            smem_attr((const void*)k_rows<T, -1>, sm);
            k_rows<T, -1><<<dim3(cdiv(nrows, NL), nsys), NTH, sm, st>>>(pl.px, (const C*)pl.twx, sys, 3, 2, nrows, NL,
                                                                         d.ex, 0, d.Lx, 0);
        }
    }, v);
}

// xoff: padded-grid index of model node 0 (1 when the convolved source lives on the extended nodes)
// dots: the systems' DotSinks receive the iteration's inner product (only on the warp-line kernel;
// the caller checks epilogue_dots_available first)
template <typename T>
static void launch_fftx_out(const Dims& d, const ApplySys<T>* sys, int nsys, const Plans& pl, int xoff, cudaStream_t st,
                            int v = 0, int dots = 0) {
    if (!fourstep_prunable(d.Lx, 0, d.nx + xoff)) v = 1;
    typedef typename cplx_of<T>::type C;
    with_engine<std::is_same<T, dfloat>::value>(d.Lx, [&](auto eng) {
        using F = decltype(eng);
        if constexpr (F::INPLACE && F::A_ == F::B_) {
            constexpr int A = F::A_, LPB = sizeof(T) == 4 ? 16 : 8;
            const long long nrows = 3LL * d.nz * d.ny;
            if constexpr (std::is_same<T, float>::value) {
                if (dots == DOT_RV) {
                    const size_t sm = (size_t)LPB * (A / 2 + 1) * A * sizeof(C);
                    smem_attr((const void*)k4_xout_w<T, A, LPB, DOT_RV>, sm, (size_t)LPB * A * (A + 1) * sizeof(C));
                    k4_xout_w<T, A, LPB, DOT_RV><<<dim3(cdiv(nrows, LPB), nsys), LPB * A, sm, st>>>(d, sys, (const C*)pl.twx,
                                                                                                   xoff);
                    return;
                }
                if (dots == DOT_TS) {
                    k4_xout_w<T, A, LPB, DOT_TS><<<dim3(cdiv(nrows, LPB), nsys), LPB * A, 0, st>>>(d, sys, (const C*)pl.twx,
                                                                                                  xoff);
                    return;
                }
            }
            k4_xout_w<T, A, LPB><<<dim3(cdiv(nrows, LPB), nsys), LPB * A, 0, st>>>(d, sys, (const C*)pl.twx, xoff);
        } else if constexpr (F::INPLACE) {
            constexpr int A = F::A_, B = F::B_, ROWS = sizeof(T) == 4 ? 8 : 4;
            const size_t sm = (size_t)A * B * (3 * ROWS + 1) * sizeof(C);
            smem_attr((const void*)k4_fftx_out<T, A, B, ROWS>, sm);
            k4_fftx_out<T, A, B, ROWS><<<dim3(cdiv(d.ny, ROWS), d.nz, nsys), 3 * ROWS * F::TPL, sm, st>>>(
                d, sys, (const C*)pl.twx, xoff);
        } else {
            int B, th;
            size_t sm;
            rows_cfg<T, F>(d.Lx, B, th, sm, v == 2);
            smem_attr((const void*)k_fftx_out<T, F>, sm);
            k_fftx_out<T, F><<<dim3(cdiv(d.ny, B), d.nz, nsys), th, sm, st>>>(d, sys, pl.px, (const C*)pl.twx, B, xoff);
        }
    }, v);
}

// Plain FFT of lines of length L along a strided axis: a.ncomp components per system, lines along
// x (a.nlines of them), `outer` line groups (blockIdx.y) per component.
template <typename T, int DIR>
static void launch_strided(int L, const FftPlan& p, const void* tw, StridedArgs a, int outer, const ApplySys<T>* sys,
                           int nsys, cudaStream_t st, int v = 0) {
    typedef typename cplx_of<T>::type C;
    if (!fourstep_prunable(L, DIR < 0 ? a.in_off + a.in_count : 0, DIR > 0 ? a.out_off + a.out_count : 0)) v = 1;
    with_engine<std::is_same<T, dfloat>::value>(L, [&](auto eng) {
        using F = decltype(eng);
        int th;
        size_t sm;
        strided_cfg<T, F>(L, 1, a.TX, th, sm, v == 2);
        if constexpr (F::INPLACE) {
            constexpr int A = F::A_, B = F::B_, TXC = sizeof(T) == 4 ? 16 : 8;
            smem_attr((const void*)k4_strided<T, DIR, A, B, TXC>, sm);
            k4_strided<T, DIR, A, B, TXC><<<dim3(cdiv(a.nlines, a.TX), outer, a.ncomp * nsys), th, sm, st>>>((const C*)tw, a, sys);
        } else {
            smem_attr((const void*)k_strided<T, DIR, F>, sm);
            k_strided<T, DIR, F><<<dim3(cdiv(a.nlines, a.TX), outer, a.ncomp * nsys), th, sm, st>>>(p, (const C*)tw, a, sys);
        }
    }, v);
}

// y pass over `planes` planes: src [ncomp][planes][in_count][Lx] (sel) -> dst [ncomp][planes][out_count][Lx] (sel)
template <typename T, int DIR>
static void launch_ypass(const Dims& d, const ApplySys<T>* sys, int nsys, const Plans& pl, int planes, int in_count,
                         int in_off, int out_count, int out_off, int src_sel, int dst_sel, cudaStream_t st, int ncomp = 3,
                         int v = 0) {
    StridedArgs a;
    a.nlines = d.Lx;
    a.in_count = in_count; a.in_off = in_off; a.out_count = out_count; a.out_off = out_off;
    a.src_es = d.Lx; a.src_os1 = (long long)in_count * d.Lx; a.src_os2 = (long long)planes * in_count * d.Lx;
    a.dst_es = d.Lx; a.dst_os1 = (long long)out_count * d.Lx; a.dst_os2 = (long long)planes * out_count * d.Lx;
    a.ncomp = ncomp; a.src_sel = src_sel; a.dst_sel = dst_sel;
    launch_strided<T, DIR>(d.Ly, pl.py, pl.twy, a, planes, sys, nsys, st, v);
}

// plain z pass: src [ncomp][in_count][Ly][Lx] (sel) -> dst [ncomp][out_count][Ly][Lx] (sel)
template <typename T, int DIR>
static void launch_zplain(const Dims& d, const ApplySys<T>* sys, int nsys, const Plans& pl, int ncomp, int in_count,
                          int out_count, int src_sel, int dst_sel, cudaStream_t st) {
    StridedArgs a;
    const long long plane = (long long)d.Ly * d.Lx;
    a.nlines = d.Lx;
    a.in_count = in_count; a.in_off = 0; a.out_count = out_count; a.out_off = 0;
    a.src_es = plane; a.src_os1 = d.Lx; a.src_os2 = (long long)in_count * plane;
    a.dst_es = plane; a.dst_os1 = d.Lx; a.dst_os2 = (long long)out_count * plane;
    a.ncomp = ncomp; a.src_sel = src_sel; a.dst_sel = dst_sel;
    launch_strided<T, DIR>(d.Lz, pl.pz, pl.twz, a, d.Ly, sys, nsys, st);
}

// schedule variant v: 0 default (register-resident kernel for FP32 and L = A * A), 1 / 2 generic
// engine (default / half tile), 3 the shared-memory four-step kernel for every precision
template <typename T, bool CONJ>
static void launch_zpass(const Dims& d, const ApplySys<T>* sys, int nsys, const Plans& pl, int in_count, int in_off,
                         int out_count, int out_off, int src_sel, int dst_sel, cudaStream_t st, int v = 0) {
    if (!fourstep_prunable(d.Lz, in_off + in_count, out_off + out_count)) v = 1;
    typedef typename cplx_of<T>::type C;
    with_engine<std::is_same<T, dfloat>::value>(d.Lz, [&](auto eng) {
        using F = decltype(eng);
        int TX, th;
        size_t sm;
        strided_cfg<T, F>(d.Lz, 3, TX, th, sm, v == 2);
        if constexpr (F::INPLACE) {
            const int E = (int)(128 / sizeof(C));
            const int GS = 6 * TX + (((TX - 6 * TX) % E) + E) % E;
            sm += (size_t)(d.nz + 1) * GS * sizeof(C);  // spectrum slice
        }
        if constexpr (F::INPLACE && sizeof(T) == 4 && F::A_ == F::B_) {
          if (v != 3) {
            constexpr int A = F::A_, TXR = 4, NL = 2 * TXR;
            constexpr int E = 16;
            constexpr int YS = A * NL + (((NL - A * NL) % E) + E) % E;
            const size_t smr = ((size_t)2 * A * YS + (size_t)6 * (d.nz + 1) * TXR + (size_t)A * A) * sizeof(C);
            smem_attr((const void*)k4z_pair<CONJ, A, TXR>, smr);
            k4z_pair<CONJ, A, TXR><<<dim3(cdiv(d.Lx, TXR), d.ny + 1, 1), 2 * TXR * A, smr, st>>>(
                d, (const float2*)pl.twz, (const ApplySys<float>*)sys, nsys, in_count, in_off, out_count, out_off,
                src_sel, dst_sel);
            return;
          }
        }
        if constexpr (F::INPLACE) {
            constexpr int A = F::A_, B = F::B_, TXC = 4;
            smem_attr((const void*)k4_fftz_green<T, CONJ, A, B, TXC>, sm);
            k4_fftz_green<T, CONJ, A, B, TXC><<<dim3(cdiv(d.Lx, TXC), d.Ly, 1), th, sm, st>>>(
                d, (const C*)pl.twz, sys, nsys, in_count, in_off, out_count, out_off, src_sel, dst_sel);
        } else {
            smem_attr((const void*)k_fftz_green<T, CONJ, F>, sm);
            k_fftz_green<T, CONJ, F><<<dim3(cdiv(d.Lx, TX), d.Ly, nsys), th, sm, st>>>(
                d, pl.pz, (const C*)pl.twz, sys, TX, in_count, in_off, out_count, out_off, src_sel, dst_sel);
        }
    }, v);
}

// ---------------------------------------------------------------------------------------------
// sampled-H form (Eq. 21 with H of Eq. 9 from the analytic derivative): the six stress planes and
// the three density terms are transformed, u-hat_i = sum_J H-hat_iJ sigma-hat_J + sum_j G-hat_ij w-hat_j
// ---------------------------------------------------------------------------------------------

// w_j = w^2 drho u_j into planes 6..8 of w1 (sigma occupies planes 0..5)
template <typename T>
__global__ void __launch_bounds__(NTH) k_hrho(Dims d, const T* __restrict__ drho, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const long long N = d.N;
    for (long long i = (long long)blockIdx.x * NTH + threadIdx.x; i < N; i += (long long)gridDim.x * NTH) {
        const T r = S.omega2 * drho[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) S.w1[(6 + c) * N + i] = cscale(S.u[c * N + i], r);
    }
}

// parity of H_iJ, J = (j, k), along axis a: odd when a occurs an odd number of times in (i, j, k)
__host__ __device__ constexpr bool h_odd(int i, int J, int a) {
    const int j = J < 3 ? J : (J == 3 ? 1 : 0);
    const int k = J < 3 ? J : (J == 5 ? 1 : 2);
    return (((i == a) + (j == a) + (k == a)) & 1) != 0;
}

// spectral product in place on w2 [9][Lz][Ly][Lx] -> planes 0..2 (each point read fully before
// it is written).  Spectra are octant-folded; a mirrored index flips the sign of the odd entries.
template <typename T>
__global__ void __launch_bounds__(NTH) k_hmul(Dims d, const ApplySys<T>* __restrict__ sys) {
    typedef typename cplx_of<T>::type C;
    const ApplySys<T> S = sys[blockIdx.y];
    if (S.run && !*S.run) return;
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    C* q = S.w2;
    const C* __restrict__ g = S.ghat;
    for (long long p = (long long)blockIdx.x * NTH + threadIdx.x; p < P; p += (long long)gridDim.x * NTH) {
        const int kx = (int)(p % d.Lx);
        const int ky = (int)((p / d.Lx) % d.Ly);
        const int kz = (int)(p / ((long long)d.Lx * d.Ly));
        const int fx = kx <= d.nx ? kx : d.Lx - kx;
        const int fy = ky <= d.ny ? ky : d.Ly - ky;
        const int fz = kz <= d.nz ? kz : d.Lz - kz;
        const unsigned m[3] = {kx > d.nx ? SIGN_BIT : 0u, ky > d.ny ? SIGN_BIT : 0u, kz > d.nz ? SIGN_BIT : 0u};
        const long long o = ((long long)fz * (d.ny + 1) + fy) * (d.nx + 1) + fx;
        C v[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) v[c] = q[c * P + p];
        const C G0 = __ldg(&g[o]), G1 = __ldg(&g[NO + o]), G2 = __ldg(&g[2 * NO + o]);
        const C G3 = flip_sign(__ldg(&g[3 * NO + o]), m[1] ^ m[2]);
        const C G4 = flip_sign(__ldg(&g[4 * NO + o]), m[0] ^ m[2]);
        const C G5 = flip_sign(__ldg(&g[5 * NO + o]), m[0] ^ m[1]);
        C out[3];
        out[0] = gdot3<false>(G0, v[6], G5, v[7], G4, v[8]);
        out[1] = gdot3<false>(G5, v[6], G1, v[7], G3, v[8]);
        out[2] = gdot3<false>(G4, v[6], G3, v[7], G2, v[8]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int J = 0; J < 6; J += 3) {
                C Hs[3];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const int JJ = J + t;
                    const unsigned mk = (h_odd(i, JJ, 0) ? m[0] : 0u) ^ (h_odd(i, JJ, 1) ? m[1] : 0u) ^
                                        (h_odd(i, JJ, 2) ? m[2] : 0u);
                    Hs[t] = flip_sign(__ldg(&g[(6 + 6 * i + JJ) * NO + o]), mk);
                }
                out[i] = cadd(out[i], gdot3<false>(Hs[0], v[J], Hs[1], v[J + 1], Hs[2], v[J + 2]));
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) q[i * P + p] = out[i];
    }
}

template <typename T>
static cudaError_t launch_apply_h(const Medium& m, const Plans& pl, const ApplySys<T>* sys, int nsys, cudaStream_t st,
                                  long long* nl) {
    typedef typename cplx_of<T>::type C;
    const Dims& d = m.d;
    KTimer* tm = m.timer;
    const bool f32 = sizeof(T) == 4;
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    // 1. stress -> w1 planes 0..5, w^2 drho u -> planes 6..8 ([9][nz][ny][nx])
    ktimer_mark(tm, 0, f32, st, 0);
    k_stress<T><<<dim3(grid_elems(d.N), nsys), NTH, 0, st>>>(d, (const T*)m.dC, sys);
    k_hrho<T><<<dim3(grid_elems(d.N), nsys), NTH, 0, st>>>(d, (const T*)m.drho, sys);
    ktimer_mark(tm, 0, f32, st, 1);
    // 2. forward x FFT of the 9 planes: w1 -> w2 [9][nz][ny][Lx]
    ktimer_mark(tm, 1, f32, st, 0);
    {
        const long long nrows = 9LL * d.nz * d.ny;
        with_engine<std::is_same<T, dfloat>::value>(d.Lx, [&](auto eng) {
            using F = decltype(eng);
            if constexpr (F::INPLACE && F::A_ == F::B_) {
                constexpr int A = F::A_, LPB = sizeof(T) == 4 ? 16 : 8;
                k4_rows_w<T, A, LPB><<<dim3(cdiv(nrows, LPB), nsys), LPB * A, 0, st>>>((const C*)pl.twx, sys, 2, 3,
                                                                                       nrows, d.nx);
            } else if constexpr (F::INPLACE) {
                constexpr int A = F::A_, B = F::B_, NL = sizeof(T) == 4 ? 8 : 12;
                const size_t sm = (size_t)A * B * (NL + 1) * sizeof(C);
                smem_attr((const void*)k4_rows<T, -1, A, B, NL>, sm);
                k4_rows<T, -1, A, B, NL><<<dim3(cdiv(nrows, NL), nsys), NL * F::TPL, sm, st>>>(
                    (const C*)pl.twx, sys, 2, 3, nrows, d.nx, 0, d.Lx, 0);
            } else {
                const int NL = generic_rows_nl<T>(d.Lx);
                const size_t sm = 2 * (size_t)d.Lx * (NL + 1) * sizeof(C);
                smem_attr((const void*)k_rows<T, -1>, sm);
                k_rows<T, -1><<<dim3(cdiv(nrows, NL), nsys), NTH, sm, st>>>(pl.px, (const C*)pl.twx, sys, 2, 3, nrows, NL,
                                                                             d.nx, 0, d.Lx, 0);
            }
        }, fourstep_prunable(d.Lx, d.nx, 0) ? 0 : 1);
    }
    ktimer_mark(tm, 1, f32, st, 1);
    // 3. forward y FFT: w2 -> w1 [9][nz][Ly][Lx]
    ktimer_mark(tm, 2, f32, st, 0);
    launch_ypass<T, -1>(d, sys, nsys, pl, d.nz, d.ny, 0, d.Ly, 0, 3, 2, st, 9);
    ktimer_mark(tm, 2, f32, st, 1);
    // 4. forward z FFT w1 -> w2 [9][Lz][Ly][Lx], spectral product in place, inverse z FFT + crop -> w1 [3][nz][Ly][Lx]
    ktimer_mark(tm, 3, f32, st, 0);
    launch_zplain<T, -1>(d, sys, nsys, pl, 9, d.nz, d.Lz, 2, 3, st);
    k_hmul<T><<<dim3(grid_elems(P), nsys), NTH, 0, st>>>(d, sys);
    launch_zplain<T, 1>(d, sys, nsys, pl, 3, d.Lz, d.nz, 3, 2, st);
    ktimer_mark(tm, 3, f32, st, 1);
    // 5. inverse y FFT + crop: w1 -> w2 [3][nz][ny][Lx]
    ktimer_mark(tm, 4, f32, st, 0);
    launch_ypass<T, 1>(d, sys, nsys, pl, d.nz, d.Ly, 0, d.ny, 0, 2, 3, st);
    ktimer_mark(tm, 4, f32, st, 1);
    // 6. inverse x FFT + crop (model node 0 at index 0) + Au = u - u_s
    ktimer_mark(tm, 5, f32, st, 0);
    launch_fftx_out<T>(d, sys, nsys, pl, 0, st, 0, std::is_same<T, float>::value ? m.dots : 0);
    ktimer_mark(tm, 5, f32, st, 1);
    if (nl) *nl += 9;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const Medium& m, const Plans& pl, const ApplySys<T>* sys, int nsys, cudaStream_t st,
                         long long* nl) {
    // the double-float operator runs the default schedule
    constexpr bool PAIR = std::is_same<T, dfloat>::value;
    if (m.kernel == 1) return launch_apply_h<T>(m, pl, sys, nsys, st, nl);
    const Dims& d = m.d;
    const T* dC = (const T*)m.dC;
    const T* drho = (const T*)m.drho;
    KTimer* tm = m.timer;
    const bool f32 = sizeof(T) == 4;
    int sched[6];
    for (int k = 0; k < 6; ++k) sched[k] = PAIR ? 0 : m.sched[k];
    if (!PAIR && sched[0] == 1) {
      if constexpr (!PAIR) {
        // 1+2. contraction fused with the divergence: q on the extended nodes -> w2 [3][ez][ey][ex]
        constexpr int TXS = 32, TYS = 8, ZC = 16;
        typedef typename cplx_of<T>::type C;
        const size_t sm = (size_t)3 * 6 * (TXS + 2) * (TYS + 2) * sizeof(C);
        smem_attr((const void*)k_sdq<T, TXS, TYS, ZC>, sm);
        ktimer_mark(tm, 0, f32, st, 0);
        k_sdq<T, TXS, TYS, ZC><<<dim3(cdiv(d.ex, TXS), cdiv(d.ey, TYS), cdiv(d.ez, ZC) * nsys), TXS * TYS, sm, st>>>(
            d, dC, drho, sys);
        ktimer_mark(tm, 0, f32, st, 1);
        ktimer_mark(tm, 1, f32, st, 0);
        launch_xfwd<T>(d, sys, nsys, pl, st, sched[1]);
        ktimer_mark(tm, 1, f32, st, 1);
        if (nl) *nl -= 1;
      }
    } else {
        // 1. strain + contraction -> w1 [6][N]
        ktimer_mark(tm, 0, f32, st, 0);
        k_stress<T><<<dim3(grid_elems(d.N), nsys), NTH, 0, st>>>(d, dC, sys);
        ktimer_mark(tm, 0, f32, st, 1);
        // 2. contrast source on the extended nodes -> w2 [3][ez][ey][ex]; forward x FFT -> w1 [3][ez][ey][Lx]
        ktimer_mark(tm, 1, f32, st, 0);
        k_divq<T><<<dim3(grid_elems((long long)d.ex * d.ey * d.ez), nsys), NTH, 0, st>>>(d, drho, sys);
        launch_xfwd<T>(d, sys, nsys, pl, st, sched[1]);
        ktimer_mark(tm, 1, f32, st, 1);
    }
    // 3. forward y FFT: w1 [3][ez][ey][Lx] -> w2 [3][ez][Ly][Lx]
    ktimer_mark(tm, 2, f32, st, 0);
    launch_ypass<T, -1>(d, sys, nsys, pl, d.ez, d.ey, 0, d.Ly, 0, 2, 3, st, 3, sched[2]);
    ktimer_mark(tm, 2, f32, st, 1);
    // 4. z FFT, Green multiply, inverse z FFT, crop: w2 [3][ez][Ly][Lx] -> w1 [3][nz][Ly][Lx]
    ktimer_mark(tm, 3, f32, st, 0);
    launch_zpass<T, false>(d, sys, nsys, pl, d.ez, 0, d.nz, 1, 3, 2, st, sched[3]);
    ktimer_mark(tm, 3, f32, st, 1);
    // 5. inverse y FFT + crop: w1 [3][nz][Ly][Lx] -> w2 [3][nz][ny][Lx]
    ktimer_mark(tm, 4, f32, st, 0);
    launch_ypass<T, 1>(d, sys, nsys, pl, d.nz, d.Ly, 0, d.ny, 1, 2, 3, st, 3, sched[4]);
    ktimer_mark(tm, 4, f32, st, 1);
    // 6. inverse x FFT + crop + Au = u - u_s (reads w2)
    ktimer_mark(tm, 5, f32, st, 0);
    launch_fftx_out<T>(d, sys, nsys, pl, 1, st, sched[5], std::is_same<T, float>::value ? m.dots : 0);
    ktimer_mark(tm, 5, f32, st, 1);
    if (nl) *nl += 7;
    return cudaGetLastError();
}

// z = K_T^H u on the extended nodes, left in w1 [3][ez][ey][ex] (the first five steps of A^H).
template <typename T>
static void launch_adjoint_conv(const Medium& m, const Plans& pl, const ApplySys<T>* sys, int nsys, cudaStream_t st) {
    typedef typename cplx_of<T>::type C;
    const Dims& d = m.d;
    const C* twx = (const C*)pl.twx;
    // 1. w placed at x positions 1..nx, forward x FFT: u [3][nz][ny][nx] -> w1 [3][nz][ny][Lx]
    {
        const int NL = generic_rows_nl<T>(d.Lx);
        const long long nrows = 3LL * d.nz * d.ny;
        const size_t sm = 2 * (size_t)d.Lx * (NL + 1) * sizeof(C);
        smem_attr((const void*)k_rows<T, -1>, sm);
        k_rows<T, -1><<<dim3(cdiv(nrows, NL), nsys), NTH, sm, st>>>(pl.px, twx, sys, 0, 2, nrows, NL, d.nx, 1, d.Lx, 0);
    }
    // 2. forward y FFT, input at 1..ny: w1 [3][nz][ny][Lx] -> w2 [3][nz][Ly][Lx]
    launch_ypass<T, -1>(d, sys, nsys, pl, d.nz, d.ny, 1, d.Ly, 0, 2, 3, st);
    // 3. z: input at 1..nz, conj(G-hat), output extended 0..ez-1: w2 -> w1 [3][ez][Ly][Lx]
    launch_zpass<T, true>(d, sys, nsys, pl, d.nz, 1, d.ez, 0, 3, 2, st);
    // 4. inverse y FFT, keep 0..ey-1: w1 [3][ez][Ly][Lx] -> w2 [3][ez][ey][Lx]
    launch_ypass<T, 1>(d, sys, nsys, pl, d.ez, d.Ly, 0, d.ey, 0, 2, 3, st);
    // 5. inverse x FFT, keep 0..ex-1: w2 [3][ez][ey][Lx] -> w1 [3][ez][ey][ex]
    {
        const int NL = generic_rows_nl<T>(d.Lx);
        const long long nrows = 3LL * d.ez * d.ey;
        const size_t sm = 2 * (size_t)d.Lx * (NL + 1) * sizeof(C);
        smem_attr((const void*)k_rows<T, 1>, sm);
        k_rows<T, 1><<<dim3(cdiv(nrows, NL), nsys), NTH, sm, st>>>(pl.px, twx, sys, 3, 2, nrows, NL, d.Lx, 0, d.ex, 0);
    }
}

template <typename T>
cudaError_t launch_adjoint(const Medium& m, const Plans& pl, const ApplySys<T>* sys, int nsys, cudaStream_t st,
                           long long* nl) {
    const Dims& d = m.d;
    const T* dC = (const T*)m.dC;
    const T* drho = (const T*)m.drho;
    launch_adjoint_conv<T>(m, pl, sys, nsys, st);
    // 6. transposed divergence + contraction -> w2 [6][N]
    k_adj_stress<T><<<dim3(grid_elems(d.N), nsys), NTH, 0, st>>>(d, dC, sys);
    // 7. transposed strain + density, AH w = w - (...)
    k_adj_out<T><<<dim3(grid_elems(d.N), nsys), NTH, 0, st>>>(d, drho, sys);
    if (nl) *nl += 7;
    return cudaGetLastError();
}

#ifndef LSM_APPLY_DFLOAT_TU
bool epilogue_dots_available(const Medium& m) {
    // the same engine choice launch_fftx_out makes: the sampled-H form crops from x offset 0 with
    // the default schedule, the difference form from offset 1 with schedule sched[5]
    const int L = m.d.Lx;
    const int xoff = m.kernel == 1 ? 0 : 1;
    const int v = m.kernel == 1 ? 0 : m.sched[5];
    return (L == 16 || L == 64 || L == 256) && v != 1 && v != 2 && fourstep_prunable(L, 0, m.d.nx + xoff);
}
int epilogue_dot_parts(const Dims& d) {
    // one partial per warp of the FP32 warp-per-line pass: 16 lines of A = sqrt(L) lanes a block
    const int A = d.Lx == 16 ? 4 : (d.Lx == 64 ? 8 : 16);
    const long long nrows = 3LL * d.nz * d.ny;
    return (int)((nrows + 15) / 16) * (16 * A / 32);
}

// Gradient of Re<lam, K_T (Dv dC eps(u) + w^2 Emb drho u)> (discrete adjoint of Eqs. 8, 11):
// z = K_T^H lam (extended nodes, in w1), tau = Dv^T z; packed entry (I, J) gets
// Re(conj(tau_I) eps_J) (+ Re(conj(tau_J) eps_I) for I != J), drho gets w^2 Re(sum_j conj(z_j) u_j).
__global__ void __launch_bounds__(NTH) k_grad(Dims d, const ApplySys<double>* __restrict__ sys, const double2* __restrict__ u,
                                              double* __restrict__ gC, double* __restrict__ grho, int accumulate) {
    typedef double2 C;
    const ApplySys<double> S = sys[0];
    const C* __restrict__ z = S.w1;
    const long long N = d.N;
    const long long E = (long long)d.ex * d.ey * d.ez;
    const double ih = 1.0 / d.h, i2h = 0.5 / d.h;
    const long long sxy = (long long)d.nx * d.ny;
    for (long long idx = (long long)blockIdx.x * NTH + threadIdx.x; idx < N; idx += (long long)gridDim.x * NTH) {
        const int ix = (int)(idx % d.nx);
        const int iy = (int)((idx / d.nx) % d.ny);
        const int iz = (int)(idx / sxy);
        auto der = [&](int c, int a) -> C {
            const C* f = u + c * N;
            const int i = a == 0 ? ix : (a == 1 ? iy : iz);
            const int n = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
            const long long s = a == 0 ? 1 : (a == 1 ? (long long)d.nx : sxy);
            if (i == 0) return cscale(csub(f[idx + s], f[idx]), ih);
            if (i == n - 1) return cscale(csub(f[idx], f[idx - s]), ih);
            return cscale(csub(f[idx + s], f[idx - s]), i2h);
        };
        C e[6];
        e[0] = der(0, 0);
        e[1] = der(1, 1);
        e[2] = der(2, 2);
        e[3] = cadd(der(1, 2), der(2, 1));
        e[4] = cadd(der(0, 2), der(2, 0));
        e[5] = cadd(der(0, 1), der(1, 0));
        const long long e0 = ((long long)(iz + 1) * d.ey + (iy + 1)) * d.ex + (ix + 1);
        const long long st[3] = {1, (long long)d.ex, (long long)d.ex * d.ey};
        C tau[6];
#pragma unroll
        for (int J = 0; J < 6; ++J) tau[J] = czero<C>();
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const C* zj = z + j * E;
                tau[t2v(j, k)] = cadd(tau[t2v(j, k)], cscale(csub(zj[e0 - st[k]], zj[e0 + st[k]]), i2h));
            }
        int k = 0;
#pragma unroll
        for (int I = 0; I < 6; ++I)
#pragma unroll
            for (int J = I; J < 6; ++J, ++k) {
                double g = tau[I].x * e[J].x + tau[I].y * e[J].y;
                if (I != J) g += tau[J].x * e[I].x + tau[J].y * e[I].y;
                double* dst = gC + (long long)k * N + idx;
                *dst = accumulate ? *dst + g : g;
            }
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const C zj = z[j * E + e0], uj = u[j * N + idx];
            r += zj.x * uj.x + zj.y * uj.y;
        }
        r *= S.omega2;
        grho[idx] = accumulate ? grho[idx] + r : r;
    }
}

cudaError_t launch_gradient(const Medium& m, const Plans& pl, const ApplySys<double>* sys, const double2* u, double* gC,
                            double* grho, int accumulate, cudaStream_t st, long long* nl) {
    launch_adjoint_conv<double>(m, pl, sys, 1, st);
    k_grad<<<grid_elems(m.d.N), NTH, 0, st>>>(m.d, sys, u, gC, grho, accumulate);
    if (nl) *nl += 6;
    return cudaGetLastError();
}

template cudaError_t launch_apply<float>(const Medium&, const Plans&, const ApplySys<float>*, int, cudaStream_t, long long*);
template cudaError_t launch_apply<double>(const Medium&, const Plans&, const ApplySys<double>*, int, cudaStream_t, long long*);
template cudaError_t launch_adjoint<double>(const Medium&, const Plans&, const ApplySys<double>*, int, cudaStream_t, long long*);
template cudaError_t launch_adjoint<float>(const Medium&, const Plans&, const ApplySys<float>*, int, cudaStream_t, long long*);

// ---------------------------------------------------------------------------------------------
// Green spectrum setup (FP64): 3-D FFT of the sampled table, in place, then octant extraction.
// ---------------------------------------------------------------------------------------------
__global__ void k_extract_octant(Dims d, const double2* __restrict__ full, double2* __restrict__ oct, double scale) {
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long total = 6 * NO;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / NO);
        long long r = i % NO;
        const int fx = (int)(r % (d.nx + 1)); r /= (d.nx + 1);
        const int fy = (int)(r % (d.ny + 1));
        const int fz = (int)(r / (d.ny + 1));
        const double2 v = full[(((long long)c * d.Lz + fz) * d.Ly + fy) * d.Lx + fx];
        oct[i] = make_double2(v.x * scale, v.y * scale);
    }
}

cudaError_t fft3_inplace_setup(const Dims& d, const Plans& pl, double2* buf, int ncomp, cudaStream_t st, long long* nl) {
    typedef double2 C;
    // x: rows
    {
        const int NL = generic_rows_nl<double>(d.Lx);
        const long long nrows = (long long)ncomp * d.Lz * d.Ly;
        const size_t sm = 2 * (size_t)d.Lx * (NL + 1) * sizeof(C);
        smem_attr((const void*)k_rows_raw<double, -1>, sm);
        k_rows_raw<double, -1><<<cdiv(nrows, NL), NTH, sm, st>>>(pl.px, (const C*)pl.twx, buf, buf, nrows, NL);
    }
    // y: lines along y, outer1 = z (Lz), comp
    {
        StridedArgs a;
        a.nlines = d.Lx; a.TX = strided_tx<double>(d.Ly, 1);
        a.in_count = d.Ly; a.in_off = 0; a.out_count = d.Ly; a.out_off = 0;
        a.src_es = d.Lx; a.src_os1 = (long long)d.Ly * d.Lx; a.src_os2 = (long long)d.Lz * d.Ly * d.Lx;
        a.dst_es = a.src_es; a.dst_os1 = a.src_os1; a.dst_os2 = a.src_os2;
        a.ncomp = ncomp; a.src_sel = a.dst_sel = 0;
        const size_t sm = 2 * (size_t)d.Ly * a.TX * sizeof(C);
        smem_attr((const void*)k_strided_raw<double, -1>, sm);
        k_strided_raw<double, -1><<<dim3(cdiv(d.Lx, a.TX), d.Lz, ncomp), NTH, sm, st>>>(pl.py, (const C*)pl.twy, a, buf, buf);
    }
    // z: lines along z, outer1 = y (Ly), comp
    {
        StridedArgs a;
        a.nlines = d.Lx; a.TX = strided_tx<double>(d.Lz, 1);
        a.in_count = d.Lz; a.in_off = 0; a.out_count = d.Lz; a.out_off = 0;
        a.src_es = (long long)d.Ly * d.Lx; a.src_os1 = d.Lx; a.src_os2 = (long long)d.Lz * d.Ly * d.Lx;
        a.dst_es = a.src_es; a.dst_os1 = a.src_os1; a.dst_os2 = a.src_os2;
        a.ncomp = ncomp; a.src_sel = a.dst_sel = 0;
        const size_t sm = 2 * (size_t)d.Lz * a.TX * sizeof(C);
        smem_attr((const void*)k_strided_raw<double, -1>, sm);
        k_strided_raw<double, -1><<<dim3(cdiv(d.Lx, a.TX), d.Ly, ncomp), NTH, sm, st>>>(pl.pz, (const C*)pl.twz, a, buf, buf);
    }
    if (nl) *nl += 3;
    return cudaGetLastError();
}

cudaError_t launch_extract_octant(const Dims& d, const double2* full, double2* oct, double scale, cudaStream_t st, long long* nl) {
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    k_extract_octant<<<grid_elems(6 * NO), NTH, 0, st>>>(d, full, oct, scale);
    if (nl) *nl += 1;
    return cudaGetLastError();
}

// Inside a stream capture the records become event-record nodes of the graph (external events),
// so every replay records the same events again.
static void ktimer_record(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}
void ktimer_mark(KTimer* t, int stage, bool f32, cudaStream_t st, int end) {
    if (!t || !t->on || !t->ev) return;
    if (!end) {
        if (t->used >= t->cap) return;
        ktimer_record(t->ev[2 * t->used], st);
        t->tag[t->used] = (f32 ? 6 : 0) + stage;
        t->open = 1;
    } else if (t->open) {
        ktimer_record(t->ev[2 * t->used + 1], st);
        t->used++;
        t->open = 0;
    }
}

// Add the recorded pairs to the totals (the caller has synchronised the stream).
void ktimer_flush(KTimer* t) {
    if (!t || !t->ev) return;
    for (int i = 0; i < t->used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t->ev[2 * i], t->ev[2 * i + 1]) == cudaSuccess) {
            t->ms[t->tag[i]] += ms;
            t->launches[t->tag[i]]++;
        }
    }
    t->used = 0;
}

cudaError_t init_kernel_attributes() {
    // dynamic shared-memory limits are raised lazily per kernel (smem_attr)
    return cudaSuccess;
}

#endif  // LSM_APPLY_DFLOAT_TU

}  // namespace lsm
