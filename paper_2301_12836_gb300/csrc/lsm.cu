// lsm.cu - host side of the C ABI declared in include/lsm.h.
//
// Handles, device memory, FFT plans and twiddle tables, and the drivers of the BiCGSTAB solve
// (Sec. 3.2): the plain FP64 solve and the mixed-precision solve (FP32 inner BiCGSTAB with FP64
// inner products, FP64 outer residual and iterative refinement).  All arithmetic of the method
// runs in the kernels of apply.cu, green.cu and solver.cu.
#include "lsm.h"
#include "kernels.h"
#include "solver.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace lsm;

namespace {

thread_local std::string g_err;

constexpr int KRY = 8;       // x, r, r^, p, v, s, t, and one scratch / inner right-hand side

struct SolverWS {
    int cap = 0;              // systems the buffers hold
    int precision = -1;
    long long n3 = 0;
    void* block = nullptr;    // one allocation for everything below
    size_t bytes = 0;
    // device arrays
    BcgState* st = nullptr;
    MixState* ms = nullptr;
    double* partials = nullptr;
    int* n_active = nullptr;
    void* vecs = nullptr;      // BcgVecs<T>[cap]
    void* sys_v = nullptr;     // ApplySys<T>[cap]
    void* sys_t = nullptr;
    void* sys_x = nullptr;
    ApplySys<double>* sys64 = nullptr;  // FP64 residual / true residual applies
    void** ptrs = nullptr;     // pointer arrays for the mix kernels: 6 * cap
    // per-system buffers (device addresses)
    std::vector<void*> kry;    // KRY Krylov vectors per system (inner precision)
    std::vector<void*> w1, w2; // inner-precision apply workspaces
    std::vector<double2*> w1d, w2d, ax64;
    std::vector<dfcplx*> xdf;  // double-float copies of the iterates (pair residual applies)
    ApplySys<dfloat>* sysdf = nullptr;
    DotSink* sinks = nullptr;  // [2][cap]: the <r^, v> and <t, s>, <t, t> sinks of the iteration applies
    float* epi = nullptr;      // [2][cap][epi_parts][4] partial sums of the epilogue inner products
    int epi_parts = 0;
    // captured BiCGSTAB iterations, one per (precision, direction); valid while block is
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int nsys = 0;
        int timer_on = 0;
        int fuse = 0;             // captured with the inner products in the apply epilogues
        long long launches = 0;   // kernels per replay
        std::vector<int> tags;    // timer slots of the captured event pairs
    } graph[2][2];                // [FP32][adjoint]
};

void drop_graphs(SolverWS& w) {
    for (auto& row : w.graph)
        for (auto& g : row) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = SolverWS::Graph();
        }
}

struct Store {
    int refs = 1;
    Dims d;
    double lam = 0, mu = 0, rho = 0;
    int precision = LSM_FP64, green = LSM_GREEN_EXACT;
    int taper = 0;
    int kernel = LSM_KERNEL_DIFF;
    int sched[2][6] = {{0}};   // FFT schedule variant per apply stage, [FP64, FP32]
    cudaStream_t st = nullptr;
    int device = 0;            // CUDA device current at lsm_create (the handle's memory lives there)
    double* dC64 = nullptr;
    double* drho64 = nullptr;
    float* dC32 = nullptr;
    float* drho32 = nullptr;
    Plans pl64, pl32, pldf;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    // double-float copies for the mixed refinement residual (LSM_RESIDUAL_DFLOAT)
    bool pair = false;
    dfloat* dCdf = nullptr;
    dfloat* drhodf = nullptr;
    dfcplx* twdf = nullptr;
    dfcplx* udf = nullptr;           // lsm_apply_df input copy
    ApplySys<dfloat>* adf = nullptr;
    // single-apply workspaces and argument slots
    double2 *w1_64 = nullptr, *w2_64 = nullptr;
    float2 *w1_32 = nullptr, *w2_32 = nullptr;
    ApplySys<double>* a64 = nullptr;
    ApplySys<float>* a32 = nullptr;
    int* flag = nullptr;
    void* h_map = nullptr;     // mapped pinned host buffer for readback() and its device alias
    void* d_map = nullptr;
    size_t map_bytes = 0;
    unsigned long long* counts = nullptr;  // device: executed system applies [FP64, FP32]
    double* grad_scratch = nullptr;        // moment-gradient partial sums
    KTimer timer;
    SolverWS ws;
    cudaStream_t cap_st = nullptr;         // private stream the iteration graphs are captured on
};

}  // namespace

struct lsm_ctx {
    Store* s = nullptr;
    double omega = 0;
    lsm_opts o;
    double2* ghat64 = nullptr;
    float2* ghat32 = nullptr;
    dfcplx* ghatdf = nullptr;
    long long nl = 0;
    std::string err;
};

namespace {

lsm_status fail(lsm_t h, lsm_status code, const std::string& msg) {
    if (h) h->err = msg; else g_err = msg;
    return code;
}

lsm_status cuda_fail(lsm_t h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LSM_ERR_OOM : LSM_ERR_CUDA, m);
}

#define CK(h, call)                                          \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #call); \
    } while (0)

bool factor_plan(int L, FftPlan& p) {
    p.L = L;
    p.nst = 0;
    int m = L;
    const int rs[5] = {8, 4, 2, 3, 5};
    for (int k = 0; k < 5; ++k) {
        while (m % rs[k] == 0) {
            if (p.nst >= 12) return false;
            p.radix[p.nst++] = rs[k];
            m /= rs[k];
        }
    }
    return m == 1;
}

// exp(-2 pi i k / L), k < L, evaluated in long double and rounded once
void twiddle_table(int L, std::vector<double2>& t64, std::vector<float2>& t32) {
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < L; ++k) {
        const long double a = -2.0L * pi * (long double)k / (long double)L;
        const long double c = cosl(a), s = sinl(a);
        t64.push_back(make_double2((double)c, (double)s));
        t32.push_back(make_float2((float)c, (float)s));
    }
}

bool lsm_grid_ok(int n) {
    if (n < 2 || 2 * n > 512) return false;
    FftPlan p;
    return factor_plan(2 * n, p);
}

void store_release(Store* s) {
    if (!s) return;
    if (--s->refs > 0) return;
    cudaFree(s->dC64); cudaFree(s->drho64); cudaFree(s->dC32); cudaFree(s->drho32);
    cudaFree(s->tw64); cudaFree(s->tw32);
    cudaFree(s->dCdf); cudaFree(s->drhodf); cudaFree(s->twdf); cudaFree(s->udf); cudaFree(s->adf);
    cudaFree(s->w1_64); cudaFree(s->w2_64); cudaFree(s->w1_32); cudaFree(s->w2_32);
    cudaFree(s->a64); cudaFree(s->a32); cudaFree(s->flag); cudaFree(s->counts); cudaFree(s->grad_scratch);
    if (s->timer.ev) {
        for (int i = 0; i < 2 * s->timer.cap; ++i) cudaEventDestroy(s->timer.ev[i]);
        delete[] s->timer.ev;
        delete[] s->timer.tag;
    }
    if (s->h_map) cudaFreeHost(s->h_map);
    drop_graphs(s->ws);
    cudaFree(s->ws.block);
    if (s->cap_st) cudaStreamDestroy(s->cap_st);
    delete s;
}

lsm_status ensure_apply_ws(lsm_t h) {
    Store* s = h->s;
    long long e1, e2;
    apply_ws_elems(s->d, s->kernel, &e1, &e2);
    if (!s->w1_64) {
        CK(h, cudaMalloc(&s->w1_64, e1 * sizeof(double2)));
        CK(h, cudaMalloc(&s->w2_64, e2 * sizeof(double2)));
    }
    if (s->precision == LSM_MIXED && !s->w1_32) {
        CK(h, cudaMalloc(&s->w1_32, e1 * sizeof(float2)));
        CK(h, cudaMalloc(&s->w2_32, e2 * sizeof(float2)));
    }
    return LSM_OK;
}

Medium medium_pair(Store* s) {
    Medium m;
    m.d = s->d;
    m.dC = s->dCdf;
    m.drho = s->drhodf;
    m.timer = &s->timer;
    m.kernel = s->kernel;
    for (int k = 0; k < 6; ++k) m.sched[k] = 0;
    return m;
}

Medium medium_of(Store* s, int prec32) {
    Medium m;
    m.d = s->d;
    m.dC = prec32 ? (const void*)s->dC32 : (const void*)s->dC64;
    m.drho = prec32 ? (const void*)s->drho32 : (const void*)s->drho64;
    m.timer = &s->timer;
    m.kernel = s->kernel;
    for (int k = 0; k < 6; ++k) m.sched[k] = s->sched[prec32 ? 1 : 0][k];
    return m;
}

// Mapped host memory for the values the host reads back while a solve runs (the source flag,
// the count of active systems, the systems' BiCGSTAB and refinement states).  A one-block kernel
// stores them there (publish) instead of a device-to-host cudaMemcpyAsync: such a copy waits in
// the copy engine's queue behind any large copy the caller has in flight on another stream
// (measured: 6.4 GB of solutions copied beside a solve stalled it for the copies' whole 33 ms
// per wave instead of overlapping).
cudaError_t map_reserve(Store* s, size_t bytes) {
    if (bytes <= s->map_bytes) return cudaSuccess;
    if (s->h_map) {
        cudaError_t e = cudaFreeHost(s->h_map);
        s->h_map = s->d_map = nullptr;
        s->map_bytes = 0;
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaHostAlloc(&s->h_map, bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        s->h_map = nullptr;
        return e;
    }
    e = cudaHostGetDevicePointer(&s->d_map, s->h_map, 0);
    if (e != cudaSuccess) return e;
    s->map_bytes = bytes;
    return cudaSuccess;
}

// Copy bytes (a multiple of 4) of device memory at dsrc to the host buffer hdst after the work
// queued on st so far; synchronizes st.
lsm_status readback(lsm_t h, const void* dsrc, void* hdst, size_t bytes, cudaStream_t st) {
    Store* s = h->s;
    CK(h, map_reserve(s, bytes));
    CK(h, publish(dsrc, s->d_map, bytes, st, &h->nl));
    CK(h, cudaStreamSynchronize(st));
    memcpy(hdst, s->h_map, bytes);
    return LSM_OK;
}

}  // namespace

extern "C" void lsm_default_opts(lsm_opts* o) {
    if (!o) return;
    o->precision = LSM_FP64;
    o->green = LSM_GREEN_EXACT;
    o->tol = 1e-10;
    o->maxit = 1000;
    o->inner_tol = 1e-6;
    o->max_outer = 8;
    o->taper = 0;
    o->graph = 1;
    o->kernel = LSM_KERNEL_DIFF;
    o->residual = LSM_RESIDUAL_FP64;
    o->fused_dots = 1;
}

static lsm_status build_spectrum(lsm_t h) {
    Store* s = h->s;
    const Dims& d = s->d;
    const long long NO = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const long long P = (long long)d.Lx * d.Ly * d.Lz;
    const long long planes = s->kernel == LSM_KERNEL_H ? 24 : 6;
    CK(h, cudaMalloc(&h->ghat64, planes * NO * sizeof(double2)));
    double2* scratch = nullptr;
    CK(h, cudaMalloc(&scratch, 6 * P * sizeof(double2)));
    cudaError_t e = launch_green_setup(d, s->pl64, s->lam, s->mu, s->rho, h->omega, s->green, s->kernel, scratch, h->ghat64,
                                       s->st, &h->nl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(h, e, "green spectrum setup");
    if (s->precision == LSM_MIXED) {
        CK(h, cudaMalloc(&h->ghat32, planes * NO * sizeof(float2)));
        CK(h, launch_d2f((const double*)h->ghat64, (float*)h->ghat32, 2 * planes * NO, s->st, &h->nl));
        CK(h, cudaStreamSynchronize(s->st));
    }
    if (s->pair) {
        CK(h, cudaMalloc(&h->ghatdf, planes * NO * sizeof(dfcplx)));
        CK(h, launch_d2df((const double*)h->ghat64, (dfloat*)h->ghatdf, 2 * planes * NO, s->st, &h->nl));
        CK(h, cudaStreamSynchronize(s->st));
    }
    return LSM_OK;
}

extern "C" lsm_status lsm_create(lsm_t* out, const int n[3], double dx, double lambda0, double mu0, double rho0,
                                 const double* dC, const double* drho, double omega, const lsm_opts* opts, void* stream) {
    if (!out) return fail(nullptr, LSM_ERR_ARG, "lsm_create: out is NULL");
    *out = nullptr;
    if (!n || !dC || !drho) return fail(nullptr, LSM_ERR_ARG, "lsm_create: null pointer argument");
    for (int a = 0; a < 3; ++a)
        if (!lsm_grid_ok(n[a]))
            return fail(nullptr, LSM_ERR_ARG, "lsm_create: each n must be >= 2 with 2n <= 512 a product of 2, 3, 5");
    if (!(dx > 0) || !(mu0 > 0) || !(lambda0 + 2 * mu0 > 0) || !(rho0 > 0) || !(omega > 0) || !std::isfinite(omega))
        return fail(nullptr, LSM_ERR_ARG, "lsm_create: need dx > 0, mu0 > 0, lambda0 + 2 mu0 > 0, rho0 > 0, omega > 0");
    lsm_opts o;
    lsm_default_opts(&o);
    if (opts) o = *opts;
    if ((o.precision != LSM_FP64 && o.precision != LSM_MIXED) || (o.green != LSM_GREEN_EXACT && o.green != LSM_GREEN_PAPER) ||
        !(o.tol > 0) || o.maxit < 1 || !(o.inner_tol > 0) || o.max_outer < 1 || o.taper < 0 ||
        (o.graph != 0 && o.graph != 1) || (o.kernel != LSM_KERNEL_DIFF && o.kernel != LSM_KERNEL_H) ||
        (o.residual != LSM_RESIDUAL_DFLOAT && o.residual != LSM_RESIDUAL_FP64) || (o.fused_dots != 0 && o.fused_dots != 1))
        return fail(nullptr, LSM_ERR_ARG, "lsm_create: invalid options");
    static bool attrs_done = false;
    if (!attrs_done) {
        cudaError_t e = init_kernel_attributes();
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "kernel attributes");
        attrs_done = true;
    }
    lsm_t h = new lsm_ctx();
    h->o = o;
    h->omega = omega;
    Store* s = new Store();
    h->s = s;
    s->st = (cudaStream_t)stream;
    if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
    s->precision = o.precision;
    s->green = o.green;
    s->pair = o.precision == LSM_MIXED && o.residual == LSM_RESIDUAL_DFLOAT;
    s->lam = lambda0; s->mu = mu0; s->rho = rho0;
    Dims& d = s->d;
    d.nx = n[0]; d.ny = n[1]; d.nz = n[2];
    d.Lx = 2 * d.nx; d.Ly = 2 * d.ny; d.Lz = 2 * d.nz;
    d.ex = d.nx + 2; d.ey = d.ny + 2; d.ez = d.nz + 2;
    d.N = (long long)d.nx * d.ny * d.nz;
    d.h = dx;
    lsm_status rc = LSM_OK;
    auto bail = [&](lsm_status r) { g_err = h->err; lsm_destroy(h); return r; };
#define CKB(call)                                                    \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return bail(cuda_fail(h, _e, #call)); \
    } while (0)
    // plans + twiddles
    {
        factor_plan(d.Lx, s->pl64.px); factor_plan(d.Ly, s->pl64.py); factor_plan(d.Lz, s->pl64.pz);
        s->pl32.px = s->pl64.px; s->pl32.py = s->pl64.py; s->pl32.pz = s->pl64.pz;
        std::vector<double2> t64;
        std::vector<float2> t32;
        twiddle_table(d.Lx, t64, t32);
        twiddle_table(d.Ly, t64, t32);
        twiddle_table(d.Lz, t64, t32);
        CKB(cudaMalloc(&s->tw64, t64.size() * sizeof(double2)));
        CKB(cudaMalloc(&s->tw32, t32.size() * sizeof(float2)));
        CKB(cudaMemcpy(s->tw64, t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice));
        CKB(cudaMemcpy(s->tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
        if (s->pair) {
            std::vector<dfcplx> tdf(t64.size());
            for (size_t i = 0; i < t64.size(); ++i) {
                tdf[i].x = dfloat(t64[i].x);
                tdf[i].y = dfloat(t64[i].y);
            }
            CKB(cudaMalloc(&s->twdf, tdf.size() * sizeof(dfcplx)));
            CKB(cudaMemcpy(s->twdf, tdf.data(), tdf.size() * sizeof(dfcplx), cudaMemcpyHostToDevice));
            s->pldf = s->pl64;
            s->pldf.twx = s->twdf; s->pldf.twy = s->twdf + d.Lx; s->pldf.twz = s->twdf + d.Lx + d.Ly;
        }
        s->pl64.twx = s->tw64; s->pl64.twy = s->tw64 + d.Lx; s->pl64.twz = s->tw64 + d.Lx + d.Ly;
        s->pl32.twx = s->tw32; s->pl32.twy = s->tw32 + d.Lx; s->pl32.twz = s->tw32 + d.Lx + d.Ly;
    }
    // contrast copies
    CKB(cudaMalloc(&s->dC64, 21 * d.N * sizeof(double)));
    CKB(cudaMalloc(&s->drho64, d.N * sizeof(double)));
    CKB(cudaMemcpyAsync(s->dC64, dC, 21 * d.N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    CKB(cudaMemcpyAsync(s->drho64, drho, d.N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    s->taper = o.taper;
    s->kernel = o.kernel;
    CKB(launch_taper(d, s->taper, s->dC64, s->drho64, s->st, &h->nl));
    if (o.precision == LSM_MIXED) {
        CKB(cudaMalloc(&s->dC32, 21 * d.N * sizeof(float)));
        CKB(cudaMalloc(&s->drho32, d.N * sizeof(float)));
        CKB(launch_d2f(s->dC64, s->dC32, 21 * d.N, s->st, &h->nl));
        CKB(launch_d2f(s->drho64, s->drho32, d.N, s->st, &h->nl));
    }
    if (s->pair) {
        CKB(cudaMalloc(&s->dCdf, 21 * d.N * sizeof(dfloat)));
        CKB(cudaMalloc(&s->drhodf, d.N * sizeof(dfloat)));
        CKB(launch_d2df(s->dC64, s->dCdf, 21 * d.N, s->st, &h->nl));
        CKB(launch_d2df(s->drho64, s->drhodf, d.N, s->st, &h->nl));
        CKB(cudaMalloc(&s->adf, sizeof(ApplySys<dfloat>)));
    }
    CKB(cudaMalloc(&s->a64, sizeof(ApplySys<double>)));
    CKB(cudaMalloc(&s->a32, sizeof(ApplySys<float>)));
    CKB(cudaMalloc(&s->flag, sizeof(int)));
    CKB(cudaMalloc(&s->counts, 2 * sizeof(unsigned long long)));
    CKB(cudaMemsetAsync(s->counts, 0, 2 * sizeof(unsigned long long), s->st));
    CKB(map_reserve(s, 4096));
    rc = build_spectrum(h);
    if (rc != LSM_OK) return bail(rc);
#undef CKB
    *out = h;
    return LSM_OK;
}

extern "C" lsm_status lsm_create_shared(lsm_t* out, lsm_t base, double omega) {
    if (!out) return fail(nullptr, LSM_ERR_ARG, "lsm_create_shared: out is NULL");
    *out = nullptr;
    if (!base) return fail(nullptr, LSM_ERR_ARG, "lsm_create_shared: base is NULL");
    if (!(omega > 0) || !std::isfinite(omega)) return fail(nullptr, LSM_ERR_ARG, "lsm_create_shared: omega must be > 0");
    lsm_t h = new lsm_ctx();
    h->o = base->o;
    h->omega = omega;
    h->s = base->s;
    h->s->refs++;
    lsm_status rc = build_spectrum(h);
    if (rc != LSM_OK) {
        g_err = h->err;
        lsm_destroy(h);
        return rc;
    }
    *out = h;
    return LSM_OK;
}

extern "C" void lsm_destroy(lsm_t h) {
    if (!h) return;
    cudaFree(h->ghat64);
    cudaFree(h->ghat32);
    cudaFree(h->ghatdf);
    store_release(h->s);
    delete h;
}

extern "C" const char* lsm_last_error(lsm_t h) {
    if (h) return h->err.c_str();
    return g_err.c_str();
}

extern "C" long long lsm_launch_count(lsm_t h) { return h ? h->nl : 0; }

static lsm_status source_fields(lsm_t h, const char* who, int nm, const double* M, const double* xs, void* const* u0) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, std::string(who) + ": null handle");
    if (!M || !xs || !u0) return fail(h, LSM_ERR_ARG, std::string(who) + ": null pointer argument");
    if (nm < 1 || nm > 4096) return fail(h, LSM_ERR_ARG, std::string(who) + ": nm must be in 1..4096");
    for (int m = 0; m < nm; ++m) {
        if (!u0[m]) return fail(h, LSM_ERR_ARG, std::string(who) + ": null output pointer");
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(M[6 * m + k])) return fail(h, LSM_ERR_ARG, std::string(who) + ": moment tensor not finite");
    }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(xs[k])) return fail(h, LSM_ERR_ARG, std::string(who) + ": source position not finite");
    Store* s = h->s;
    CK(h, cudaMemsetAsync(s->flag, 0, sizeof(int), s->st));
    CK(h, launch_source(s->d, s->lam, s->mu, s->rho, h->omega, s->green, nm, M, xs, (double2* const*)u0, s->flag, s->st,
                        &h->nl));
    int on_node = 0;
    lsm_status rb = readback(h, s->flag, &on_node, sizeof(int), s->st);
    if (rb != LSM_OK) return rb;
    if (on_node) {
        h->err = std::string(who) + ": a grid node coincides with the source; u0 set to 0 there";
        return LSM_WARN_SOURCE_ON_NODE;
    }
    return LSM_OK;
}

extern "C" lsm_status lsm_source(lsm_t h, const double M[6], const double xs[3], void* u0) {
    void* out[1] = {u0};
    return source_fields(h, "lsm_source", 1, M, xs, out);
}

extern "C" lsm_status lsm_source_moments(lsm_t h, int nm, const double* M, const double xs[3], void* const* u0) {
    return source_fields(h, "lsm_source_moments", nm, M, xs, u0);
}

template <typename T>
static lsm_status apply_one(lsm_t h, const void* u, void* Au, bool adjoint) {
    typedef typename cplx_of<T>::type C;
    Store* s = h->s;
    lsm_status rc = ensure_apply_ws(h);
    if (rc != LSM_OK) return rc;
    const bool f32 = sizeof(T) == 4;
    ApplySys<T> a;
    a.u = (const C*)u;
    a.out = (C*)Au;
    a.ghat = f32 ? (const C*)h->ghat32 : (const C*)h->ghat64;
    a.w1 = f32 ? (C*)s->w1_32 : (C*)s->w1_64;
    a.w2 = f32 ? (C*)s->w2_32 : (C*)s->w2_64;
    a.omega2 = (T)(h->omega * h->omega);
    a.run = nullptr;
    a.count = s->counts + (f32 ? 1 : 0);
    ApplySys<T>* dev = f32 ? (ApplySys<T>*)s->a32 : (ApplySys<T>*)s->a64;
    CK(h, cudaMemcpyAsync(dev, &a, sizeof(a), cudaMemcpyHostToDevice, s->st));
    const Plans& pl = f32 ? s->pl32 : s->pl64;
    Medium m = medium_of(s, f32);
    cudaError_t e = adjoint ? launch_adjoint<T>(m, pl, dev, 1, s->st, &h->nl) : launch_apply<T>(m, pl, dev, 1, s->st, &h->nl);
    if (e != cudaSuccess) return cuda_fail(h, e, adjoint ? "adjoint" : "apply");
    return LSM_OK;
}

extern "C" lsm_status lsm_apply(lsm_t h, const void* u, void* Au) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_apply: null handle");
    if (!u || !Au || u == Au) return fail(h, LSM_ERR_ARG, "lsm_apply: u and Au must be distinct non-null device buffers");
    return apply_one<double>(h, u, Au, false);
}

extern "C" lsm_status lsm_apply_c64(lsm_t h, const void* u, void* Au) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_apply_c64: null handle");
    if (!u || !Au || u == Au) return fail(h, LSM_ERR_ARG, "lsm_apply_c64: u and Au must be distinct non-null device buffers");
    if (h->s->precision != LSM_MIXED) return fail(h, LSM_ERR_ARG, "lsm_apply_c64: handle was not created with LSM_MIXED");
    return apply_one<float>(h, u, Au, false);
}

extern "C" lsm_status lsm_apply_df(lsm_t h, const void* u, void* Au) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_apply_df: null handle");
    if (!u || !Au || u == Au) return fail(h, LSM_ERR_ARG, "lsm_apply_df: u and Au must be distinct non-null device buffers");
    Store* s = h->s;
    if (!s->pair)
        return fail(h, LSM_ERR_ARG, "lsm_apply_df: needs a handle created with LSM_MIXED and LSM_RESIDUAL_DFLOAT");
    lsm_status rc = ensure_apply_ws(h);
    if (rc != LSM_OK) return rc;
    const long long n3 = 3 * s->d.N;
    if (!s->udf) CK(h, cudaMalloc(&s->udf, n3 * sizeof(dfcplx)));
    CK(h, launch_d2df((const double*)u, (dfloat*)s->udf, 2 * n3, s->st, &h->nl));
    ApplySys<dfloat> a;
    a.u = s->udf;
    a.out = (dfcplx*)Au;
    a.ghat = h->ghatdf;
    a.w1 = (dfcplx*)s->w1_64;
    a.w2 = (dfcplx*)s->w2_64;
    a.omega2 = dfloat(h->omega * h->omega);
    a.run = nullptr;
    a.count = s->counts;
    CK(h, cudaMemcpyAsync(s->adf, &a, sizeof(a), cudaMemcpyHostToDevice, s->st));
    cudaError_t e = launch_apply<dfloat>(medium_pair(s), s->pldf, s->adf, 1, s->st, &h->nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "lsm_apply_df");
    CK(h, launch_df2d_inplace(Au, 2 * n3, s->st, &h->nl));
    return LSM_OK;
}

extern "C" lsm_status lsm_adjoint(lsm_t h, const void* v, void* AHv) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_adjoint: null handle");
    if (!v || !AHv || v == AHv) return fail(h, LSM_ERR_ARG, "lsm_adjoint: v and AHv must be distinct non-null device buffers");
    if (h->s->kernel == LSM_KERNEL_H) return fail(h, LSM_ERR_ARG, "lsm_adjoint: not available for LSM_KERNEL_H");
    return apply_one<double>(h, v, AHv, true);
}

// ---------------------------------------------------------------------------------------------
// solver workspace
// ---------------------------------------------------------------------------------------------
namespace {

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int GRAPH_ITERS = 2;   // BiCGSTAB iterations per captured graph

lsm_status ensure_solver_ws(lsm_t h, int nsys) {
    Store* s = h->s;
    SolverWS& w = s->ws;
    const long long n3 = 3 * s->d.N;
    if (w.cap >= nsys && w.precision == s->precision) return LSM_OK;
    drop_graphs(w);
    cudaFree(w.block);
    w = SolverWS();
    long long e1, e2;
    apply_ws_elems(s->d, s->kernel, &e1, &e2);
    const bool mixed = s->precision == LSM_MIXED;
    const size_t csz = mixed ? sizeof(float2) : sizeof(double2);
    const int nblk = vec_blocks(n3);
    // layout
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
    const size_t o_st = take(nsys * sizeof(BcgState));
    const size_t o_ms = take(nsys * sizeof(MixState));
    const size_t o_pt = take((size_t)nsys * nblk * 4 * sizeof(double));
    const size_t o_na = take(sizeof(int));
    const size_t o_vecs = take(nsys * sizeof(BcgVecs<double>));
    const size_t o_sv = take(nsys * sizeof(ApplySys<double>));
    const size_t o_stt = take(nsys * sizeof(ApplySys<double>));
    const size_t o_sx = take(nsys * sizeof(ApplySys<double>));
    const size_t o_s64 = take(nsys * sizeof(ApplySys<double>));
    const size_t o_ptr = take(7 * (size_t)nsys * sizeof(void*));
    const size_t o_sdf = take(nsys * sizeof(ApplySys<dfloat>));
    const int epi_parts = epilogue_dot_parts(s->d);
    const size_t o_snk = take(2 * (size_t)nsys * sizeof(DotSink));
    const size_t o_epi = take(2 * (size_t)nsys * epi_parts * 4 * sizeof(float));
    std::vector<size_t> o_kry, o_w1, o_w2, o_w1d, o_w2d, o_ax, o_xdf;
    for (int i = 0; i < nsys; ++i) {
        for (int k = 0; k < KRY; ++k) o_kry.push_back(take(n3 * csz));
        if (mixed) {
            // FP64 residual-apply workspaces; the FP32 inner ones alias their first halves
            // (the FP64 apply and the inner solve never run at the same time)
            o_w1d.push_back(take(e1 * sizeof(double2)));
            o_w2d.push_back(take(e2 * sizeof(double2)));
            o_ax.push_back(take(n3 * sizeof(double2)));
            if (s->pair) o_xdf.push_back(take(n3 * sizeof(dfcplx)));
        } else {
            o_w1.push_back(take(e1 * csz));
            o_w2.push_back(take(e2 * csz));
        }
    }
    w.bytes = off;
    cudaError_t e = cudaMalloc(&w.block, off);
    if (e != cudaSuccess) {
        w = SolverWS();
        return cuda_fail(h, e, "solver workspace");
    }
    char* b = (char*)w.block;
    // readbacks of the systems' states go through the mapped buffer: size it for this batch now
    const size_t state_bytes = sizeof(BcgState) > sizeof(MixState) ? sizeof(BcgState) : sizeof(MixState);
    CK(h, map_reserve(s, (size_t)nsys * state_bytes + 256));
    w.cap = nsys;
    w.precision = s->precision;
    w.n3 = n3;
    w.st = (BcgState*)(b + o_st);
    w.ms = (MixState*)(b + o_ms);
    w.partials = (double*)(b + o_pt);
    w.n_active = (int*)(b + o_na);
    w.vecs = b + o_vecs;
    w.sys_v = b + o_sv;
    w.sys_t = b + o_stt;
    w.sys_x = b + o_sx;
    w.sys64 = (ApplySys<double>*)(b + o_s64);
    w.ptrs = (void**)(b + o_ptr);
    w.sysdf = (ApplySys<dfloat>*)(b + o_sdf);
    w.sinks = (DotSink*)(b + o_snk);
    w.epi = (float*)(b + o_epi);
    w.epi_parts = epi_parts;
    for (int i = 0; i < nsys; ++i) {
        for (int k = 0; k < KRY; ++k) w.kry.push_back(b + o_kry[i * KRY + k]);
        if (mixed) {
            w.w1d.push_back((double2*)(b + o_w1d[i]));
            w.w2d.push_back((double2*)(b + o_w2d[i]));
            w.w1.push_back(b + o_w1d[i]);
            w.w2.push_back(b + o_w2d[i]);
            w.ax64.push_back((double2*)(b + o_ax[i]));
            if (s->pair) w.xdf.push_back((dfcplx*)(b + o_xdf[i]));
        } else {
            w.w1.push_back(b + o_w1[i]);
            w.w2.push_back(b + o_w2[i]);
        }
    }
    return LSM_OK;
}

}  // namespace

lsm_status tune_workspace(lsm_t h, int nsys) { return ensure_solver_ws(h, nsys); }

namespace {

// A (adjoint = false) or A^H (adjoint = true) for nsys systems
template <typename T>
cudaError_t apply_op(bool adjoint, const Medium& m, const Plans& pl, const ApplySys<T>* sys, int nsys, cudaStream_t st,
                     long long* nl) {
    return adjoint ? launch_adjoint<T>(m, pl, sys, nsys, st, nl) : launch_apply<T>(m, pl, sys, nsys, st, nl);
}

// Run BiCGSTAB on nsys systems whose vectors/apply arguments are already on the device.
// fuse: the iteration applies' epilogues sum <r^, v> and <t, s>, <t, t> (their ApplySys::dot are
// set) and dot_finish, one block per system, finishes alpha and omega from their partial sums in
// place of the two vector kernels that would read the vectors again
template <typename T>
lsm_status run_bicgstab(lsm_t h0, const std::vector<lsm_t>& hs, int nsys, const std::vector<double>& tol, int maxit,
                        bool x_zero, const MixState* skip, std::vector<BcgState>& out, bool adjoint, bool fuse) {
    Store* s = h0->s;
    SolverWS& w = s->ws;
    const long long n3 = w.n3;
    const cudaStream_t st = s->st;
    Partials pt;
    pt.buf = w.partials;
    pt.nblk = vec_blocks(n3);
    BcgVecs<T>* vecs = (BcgVecs<T>*)w.vecs;
    ApplySys<T>* sv = (ApplySys<T>*)w.sys_v;
    ApplySys<T>* stt = (ApplySys<T>*)w.sys_t;
    ApplySys<T>* sx = (ApplySys<T>*)w.sys_x;
    const bool f32 = sizeof(T) == 4;
    const Plans& pl = f32 ? s->pl32 : s->pl64;
    Medium m = medium_of(s, f32);
    long long* nl = &h0->nl;
    std::vector<BcgState> init(nsys);
    for (int i = 0; i < nsys; ++i) {
        BcgState& b = init[i];
        memset(&b, 0, sizeof(b));
        b.tol2 = tol[i] * tol[i];
        b.maxit = maxit;
        b.active = 0;
    }
    CK(h0, cudaMemcpyAsync(w.st, init.data(), nsys * sizeof(BcgState), cudaMemcpyHostToDevice, st));
    CK(h0, cudaMemsetAsync(w.n_active, 0, sizeof(int), st));
    if (!x_zero) {
        cudaError_t e = apply_op<T>(adjoint, m, pl, sx, nsys, st, nl);
        if (e != cudaSuccess) return cuda_fail(h0, e, "initial residual apply");
    }
    CK(h0, bcg_init<T>(vecs, w.st, pt, n3, nsys, x_zero ? 1 : 0, skip, w.n_active, st, nl));
    int n_active = 0;
    lsm_status rb = readback(h0, w.n_active, &n_active, sizeof(int), st);
    if (rb != LSM_OK) return rb;
    // one iteration for every system on stream q; kernels of systems that stopped return at once
    Medium mv = m, mt = m;
    mv.dots = fuse ? DOT_RV : 0;
    mt.dots = fuse ? DOT_TS : 0;
    auto iterate = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = bcg_update_p<T>(vecs, w.st, n3, nsys, pt.nblk, q, nl);
        if (e == cudaSuccess) e = apply_op<T>(adjoint, mv, pl, sv, nsys, q, nl);
        if (e == cudaSuccess) e = fuse ? dot_finish(w.sinks, nsys, q, nl) : bcg_alpha<T>(vecs, w.st, pt, n3, nsys, w.n_active, q, nl);
        if (e == cudaSuccess) e = bcg_s<T>(vecs, w.st, pt, n3, nsys, q, nl);
        if (e == cudaSuccess) e = apply_op<T>(adjoint, mt, pl, stt, nsys, q, nl);
        if (e == cudaSuccess) e = fuse ? dot_finish(w.sinks + nsys, nsys, q, nl) : bcg_omega<T>(vecs, w.st, pt, n3, nsys, q, nl);
        if (e == cudaSuccess) e = bcg_xr<T>(vecs, w.st, pt, n3, nsys, w.n_active, q, nl);
        return e;
    };
    const bool use_graph = h0->o.graph != 0;
    SolverWS::Graph& G = w.graph[f32 ? 1 : 0][adjoint ? 1 : 0];
    KTimer& tm = s->timer;
    int done = 0;   // iterations issued (each system also counts its own and stops at maxit)
    while (n_active > 0 && done <= maxit + 1) {
        if (!use_graph || done == 0) {
            // eager: always the first iteration, so every kernel is loaded and configured
            // before a capture
            cudaError_t e = iterate(st);
            if (e != cudaSuccess) return cuda_fail(h0, e, "BiCGSTAB iteration");
            done += 1;
        } else {
            const int tm_on = (tm.on && tm.ev) ? 1 : 0;
            if (G.exec && (G.nsys != nsys || G.timer_on != tm_on || G.fuse != (fuse ? 1 : 0))) {
                cudaGraphExecDestroy(G.exec);
                G = SolverWS::Graph();
            }
            if (!G.exec) {
                // captured on a private stream (the caller's may be the legacy default stream,
                // which cannot be captured); replayed on the caller's
                if (!s->cap_st) CK(h0, cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
                const long long nl0 = *nl;
                tm.used = 0;
                tm.open = 0;
                CK(h0, cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = cudaSuccess;
                for (int k = 0; k < GRAPH_ITERS && e == cudaSuccess; ++k) e = iterate(s->cap_st);
                cudaGraph_t g = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(s->cap_st, &g);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
                if (g) cudaGraphDestroy(g);
                // the launchers counted the captured kernels: that is the count of one replay
                const long long captured = *nl - nl0;
                *nl = nl0;
                if (e != cudaSuccess) {
                    G = SolverWS::Graph();
                    tm.used = 0;
                    return cuda_fail(h0, e, "BiCGSTAB iteration graph");
                }
                G.nsys = nsys;
                G.timer_on = tm_on;
                G.fuse = fuse ? 1 : 0;
                G.launches = captured;
                G.tags.assign(tm.tag, tm.tag + tm.used);
                tm.used = 0;
            }
            CK(h0, cudaGraphLaunch(G.exec, st));
            *nl += G.launches;
            if (tm_on) {
                std::copy(G.tags.begin(), G.tags.end(), tm.tag);
                tm.used = (int)G.tags.size();
            }
            done += GRAPH_ITERS;
        }
        if ((rb = readback(h0, w.n_active, &n_active, sizeof(int), st)) != LSM_OK) return rb;
        ktimer_flush(&tm);
    }
    out.resize(nsys);
    return readback(h0, w.st, out.data(), nsys * sizeof(BcgState), st);
}

}  // namespace

// Point the iteration applies of the nsys systems at their DotSinks: v = A p sums <r^, v> into
// sink i, t = A s sums <t, s> and <t, t> into sink nsys + i (each with its own partial sums).
template <typename T, typename C>
static lsm_status set_dot_sinks(lsm_t h0, int nsys, const std::vector<BcgVecs<C>>& V, std::vector<ApplySys<T>>& sv,
                                std::vector<ApplySys<T>>& stt) {
    SolverWS& w = h0->s->ws;
    std::vector<DotSink> dk(2 * (size_t)nsys);
    for (int i = 0; i < nsys; ++i) {
        for (int k = 0; k < 2; ++k) {
            DotSink& q = dk[(size_t)k * nsys + i];
            q.st = &w.st[i];
            q.rh = k == 0 ? (const void*)V[i].rh : nullptr;
            q.partials = w.epi + ((size_t)k * nsys + i) * w.epi_parts * 4;
            q.nparts = w.epi_parts;
            q.mode = k == 0 ? DOT_RV : DOT_TS;
            q.n_active = w.n_active;
        }
        sv[i].dot = w.sinks + i;
        stt[i].dot = w.sinks + nsys + i;
    }
    CK(h0, cudaMemcpyAsync(w.sinks, dk.data(), dk.size() * sizeof(DotSink), cudaMemcpyHostToDevice, h0->s->st));
    return LSM_OK;
}

static lsm_status solve_batched(int nsys, const lsm_t* hs_in, const void* const* b, void* const* x, int* iters,
                                double* relres, lsm_status* status, bool adjoint) {
    if (nsys < 1 || !hs_in || !b || !x) return fail(nullptr, LSM_ERR_ARG, "lsm_solve_batched: bad arguments");
    std::vector<lsm_t> hs(hs_in, hs_in + nsys);
    for (int i = 0; i < nsys; ++i) {
        if (!hs[i]) return fail(nullptr, LSM_ERR_ARG, "lsm_solve_batched: null handle");
        if (hs[i]->s != hs[0]->s) return fail(hs[0], LSM_ERR_ARG, "lsm_solve_batched: handles must share one medium");
        if (!b[i] || !x[i] || b[i] == x[i]) return fail(hs[0], LSM_ERR_ARG, "lsm_solve_batched: b and x must be distinct device buffers");
    }
    lsm_t h0 = hs[0];
    Store* s = h0->s;
    const cudaStream_t st = s->st;
    lsm_status rc = ensure_solver_ws(h0, nsys);
    if (rc != LSM_OK) return rc;
    SolverWS& w = s->ws;
    const long long n3 = w.n3;
    const bool mixed = s->precision == LSM_MIXED;
    const double tol = h0->o.tol;
    Partials pt;
    pt.buf = w.partials;
    pt.nblk = vec_blocks(n3);
    std::vector<int> it_out(nsys, 0);
    std::vector<double> rr_out(nsys, 0.0);
    std::vector<lsm_status> stat(nsys, LSM_OK);
    // final-residual / FP64 apply arguments
    std::vector<ApplySys<double>> a64(nsys);
    std::vector<MixState> ms(nsys);
    for (int i = 0; i < nsys; ++i) {
        memset(&ms[i], 0, sizeof(MixState));
        ms[i].tol = tol;
    }
    if (!mixed) {
        std::vector<BcgVecs<double>> V(nsys);
        std::vector<ApplySys<double>> sv(nsys), stt(nsys), sx(nsys);
        for (int i = 0; i < nsys; ++i) {
            double2** k = (double2**)&w.kry[i * KRY];
            V[i].b = (const double2*)b[i];
            V[i].x = (double2*)x[i];
            V[i].r = k[0]; V[i].rh = k[1]; V[i].p = k[2]; V[i].v = k[3]; V[i].s = k[4]; V[i].t = k[5];
            ApplySys<double> a;
            a.count = s->counts;
            a.ghat = hs[i]->ghat64;
            a.w1 = (double2*)w.w1[i];
            a.w2 = (double2*)w.w2[i];
            a.omega2 = hs[i]->omega * hs[i]->omega;
            a.u = V[i].p; a.out = V[i].v; a.run = &w.st[i].run_v; sv[i] = a;
            a.u = V[i].s; a.out = V[i].t; a.run = &w.st[i].run_t; stt[i] = a;
            a.u = V[i].x; a.out = V[i].v; a.run = nullptr; sx[i] = a;
            a.u = V[i].x; a.out = k[6]; a.run = nullptr; a64[i] = a;   // true residual at exit
        }
        // FP64 iterations keep the vector kernels: the FP64 epilogue is bound by the FP64 pipe,
        // so the same FP64 products cost it as much as a separate kernel that streams the vectors
        const bool fuse = false;
        CK(h0, cudaMemcpyAsync(w.vecs, V.data(), nsys * sizeof(V[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys_v, sv.data(), nsys * sizeof(sv[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys_t, stt.data(), nsys * sizeof(stt[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys_x, sx.data(), nsys * sizeof(sx[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys64, a64.data(), nsys * sizeof(a64[0]), cudaMemcpyHostToDevice, st));
        std::vector<BcgState> fin;
        rc = run_bicgstab<double>(h0, hs, nsys, std::vector<double>(nsys, tol), h0->o.maxit, false, nullptr, fin, adjoint,
                                  fuse);
        if (rc != LSM_OK) return rc;
        for (int i = 0; i < nsys; ++i) {
            it_out[i] = fin[i].iters;
            stat[i] = (lsm_status)fin[i].status;
            // b = 0: the solution is exactly zero whatever the initial guess
            if (fin[i].bnorm2 == 0.0) CK(h0, cudaMemsetAsync(x[i], 0, n3 * sizeof(double2), st));
        }
        // true residual ||b - A x|| / ||b|| (Eq. 22)
        Medium m = medium_of(s, 0);
        cudaError_t e = apply_op<double>(adjoint, m, s->pl64, w.sys64, nsys, st, &h0->nl);
        if (e != cudaSuccess) return cuda_fail(h0, e, "final residual apply");
        void** P = w.ptrs;
        std::vector<void*> hp(6 * nsys);
        for (int i = 0; i < nsys; ++i) {
            hp[i] = const_cast<void*>(b[i]);
            hp[nsys + i] = w.kry[i * KRY + 6];
            hp[2 * nsys + i] = w.kry[i * KRY + 7];   // residual scratch
        }
        CK(h0, cudaMemcpyAsync(P, hp.data(), 6 * nsys * sizeof(void*), cudaMemcpyHostToDevice, st));
        ms.assign(nsys, MixState());
        for (int i = 0; i < nsys; ++i) { memset(&ms[i], 0, sizeof(MixState)); ms[i].tol = 0.0; }
        CK(h0, cudaMemcpyAsync(w.ms, ms.data(), nsys * sizeof(MixState), cudaMemcpyHostToDevice, st));
        CK(h0, mix_residual((const double2* const*)P, (const double2* const*)(P + nsys), (double2* const*)(P + 2 * nsys), w.ms, pt,
                            n3, nsys, w.n_active, st, &h0->nl));
        if ((rc = readback(h0, w.ms, ms.data(), nsys * sizeof(MixState), st)) != LSM_OK) return rc;
        for (int i = 0; i < nsys; ++i) rr_out[i] = ms[i].relres;
    } else {
        // mixed precision: outer residual in double-float (pair) or FP64 arithmetic, FP64 storage, and
        // FP32 inner BiCGSTAB on the normalised residual
        const bool pair = s->pair && !adjoint;
        std::vector<ApplySys<dfloat>> adf(nsys);
        std::vector<BcgVecs<float>> V(nsys);
        std::vector<ApplySys<float>> sv(nsys), stt(nsys);
        for (int i = 0; i < nsys; ++i) {
            float2** k = (float2**)&w.kry[i * KRY];
            V[i].x = k[0];   // correction d
            V[i].r = k[1]; V[i].rh = k[2]; V[i].p = k[3]; V[i].v = k[4]; V[i].s = k[5]; V[i].t = k[6];
            V[i].b = k[7];   // normalised FP32 residual
            ApplySys<float> a;
            a.count = s->counts + 1;
            a.ghat = hs[i]->ghat32;
            a.w1 = (float2*)w.w1[i];
            a.w2 = (float2*)w.w2[i];
            a.omega2 = (float)(hs[i]->omega * hs[i]->omega);
            a.u = V[i].p; a.out = V[i].v; a.run = &w.st[i].run_v; sv[i] = a;
            a.u = V[i].s; a.out = V[i].t; a.run = &w.st[i].run_t; stt[i] = a;
            ApplySys<double> d;
            d.count = s->counts;
            d.ghat = hs[i]->ghat64;
            d.w1 = w.w1d[i];
            d.w2 = w.w2d[i];
            d.omega2 = hs[i]->omega * hs[i]->omega;
            d.u = (const double2*)x[i];
            d.out = w.ax64[i];
            d.run = &w.ms[i].run;
            a64[i] = d;
            if (pair) {
                ApplySys<dfloat> q;
                q.count = s->counts;
                q.ghat = hs[i]->ghatdf;
                q.w1 = (dfcplx*)w.w1d[i];
                q.w2 = (dfcplx*)w.w2d[i];
                q.omega2 = dfloat(hs[i]->omega * hs[i]->omega);
                q.u = w.xdf[i];
                q.out = (dfcplx*)w.ax64[i];   // A x as pairs, read back by the pair residual
                q.run = &w.ms[i].run;
                adf[i] = q;
            }
        }
        const bool fuse = !adjoint && h0->o.fused_dots && epilogue_dots_available(medium_of(s, 1));
        if (fuse && (rc = set_dot_sinks(h0, nsys, V, sv, stt)) != LSM_OK) return rc;
        if (pair) CK(h0, cudaMemcpyAsync(w.sysdf, adf.data(), nsys * sizeof(adf[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.vecs, V.data(), nsys * sizeof(V[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys_v, sv.data(), nsys * sizeof(sv[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys_t, stt.data(), nsys * sizeof(stt[0]), cudaMemcpyHostToDevice, st));
        CK(h0, cudaMemcpyAsync(w.sys64, a64.data(), nsys * sizeof(a64[0]), cudaMemcpyHostToDevice, st));
        void** P = w.ptrs;
        std::vector<void*> hp(7 * nsys, nullptr);
        for (int i = 0; i < nsys; ++i) {
            hp[i] = const_cast<void*>(b[i]);
            hp[nsys + i] = w.ax64[i];
            hp[2 * nsys + i] = w.ax64[i];     // r64 overwrites ax64 in place
            hp[3 * nsys + i] = w.kry[i * KRY + 7];  // r32 (inner b)
            hp[4 * nsys + i] = x[i];
            hp[5 * nsys + i] = w.kry[i * KRY + 0];  // d32
            if (pair) hp[6 * nsys + i] = w.xdf[i];
        }
        CK(h0, cudaMemcpyAsync(P, hp.data(), 7 * nsys * sizeof(void*), cudaMemcpyHostToDevice, st));
        for (int i = 0; i < nsys; ++i) ms[i].run = 1;
        CK(h0, cudaMemcpyAsync(w.ms, ms.data(), nsys * sizeof(MixState), cudaMemcpyHostToDevice, st));
        // a zero initial guess needs no FP64 apply: its residual is b
        CK(h0, mix_xnorm((const double2* const*)(P + 4 * nsys), w.ms, pt, n3, nsys, st, &h0->nl));
        Medium m64 = medium_of(s, 0);
        const int nblk = pt.nblk;
        std::vector<double> itol(nsys, h0->o.inner_tol);
        for (int outer = 0;; ++outer) {
            cudaError_t e;
            if (pair) {
                CK(h0, mix_to_pair((const double2* const*)(P + 4 * nsys), (dfcplx* const*)(P + 6 * nsys), w.ms, n3, nsys, nblk,
                                   st, &h0->nl));
                e = launch_apply<dfloat>(medium_pair(s), s->pldf, w.sysdf, nsys, st, &h0->nl);
            } else {
                e = apply_op<double>(adjoint, m64, s->pl64, w.sys64, nsys, st, &h0->nl);
            }
            if (e != cudaSuccess) return cuda_fail(h0, e, "residual apply");
            CK(h0, cudaMemsetAsync(w.n_active, 0, sizeof(int), st));
            CK(h0, mix_residual((const double2* const*)P, (const double2* const*)(P + nsys), (double2* const*)(P + 2 * nsys), w.ms,
                                pt, n3, nsys, w.n_active, st, &h0->nl, pair));
            if ((rc = readback(h0, w.ms, ms.data(), nsys * sizeof(MixState), st)) != LSM_OK) return rc;
            ktimer_flush(&s->timer);
            int n_act = 0;
            for (int i = 0; i < nsys; ++i) n_act += !ms[i].done;
            if (n_act == 0 || outer >= h0->o.max_outer) break;
            // each inner FP32 solve aims a decade below what the outer target still needs,
            // never tighter than inner_tol (the floor FP32 arithmetic can certify)
            for (int i = 0; i < nsys; ++i) {
                const double need = ms[i].relres > 0 ? 0.1 * tol / ms[i].relres : 1.0;
                itol[i] = need < h0->o.inner_tol ? h0->o.inner_tol : (need > 0.1 ? 0.1 : need);
            }
            CK(h0, mix_down((double2* const*)(P + 2 * nsys), (float2* const*)(P + 3 * nsys), w.ms, n3, nsys, nblk, st, &h0->nl));
            for (int i = 0; i < nsys; ++i) CK(h0, cudaMemsetAsync(w.kry[i * KRY + 0], 0, n3 * sizeof(float2), st));
            std::vector<BcgState> fin;
            rc = run_bicgstab<float>(h0, hs, nsys, itol, h0->o.maxit, true, w.ms, fin, adjoint, fuse);
            if (rc != LSM_OK) return rc;
            for (int i = 0; i < nsys; ++i) it_out[i] += fin[i].iters;
            CK(h0, mix_up((double2* const*)(P + 4 * nsys), (float2* const*)(P + 5 * nsys), w.ms, w.st, n3, nsys, nblk, st,
                          &h0->nl));
        }
        if ((rc = readback(h0, w.ms, ms.data(), nsys * sizeof(MixState), st)) != LSM_OK) return rc;
        for (int i = 0; i < nsys; ++i) {
            rr_out[i] = ms[i].relres;
            stat[i] = (ms[i].done && !ms[i].stalled) ? LSM_OK : LSM_ERR_NOCONV;
            if (ms[i].bnorm2 == 0.0) CK(h0, cudaMemsetAsync(x[i], 0, n3 * sizeof(double2), st));
        }
        CK(h0, cudaStreamSynchronize(st));
    }
    lsm_status first = LSM_OK;
    for (int i = 0; i < nsys; ++i) {
        if (iters) iters[i] = it_out[i];
        if (relres) relres[i] = rr_out[i];
        if (status) status[i] = stat[i];
        if (stat[i] != LSM_OK && first == LSM_OK) first = stat[i];
    }
    if (first != LSM_OK) h0->err = first == LSM_ERR_NOCONV ? "solve: iteration limit reached" : "solve: BiCGSTAB breakdown";
    return first;
}

extern "C" lsm_status lsm_solve_batched(int nsys, const lsm_t* hs, const void* const* b, void* const* x, int* iters,
                                        double* relres, lsm_status* status) {
    return solve_batched(nsys, hs, b, x, iters, relres, status, false);
}

extern "C" lsm_status lsm_solve(lsm_t h, const void* b, void* x, int* iters, double* relres) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_solve: null handle");
    const void* bb[1] = {b};
    void* xx[1] = {x};
    return solve_batched(1, &h, bb, xx, iters, relres, nullptr, false);
}

extern "C" lsm_status lsm_solve_adjoint(lsm_t h, const void* b, void* x, int* iters, double* relres) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_solve_adjoint: null handle");
    if (h->s->kernel == LSM_KERNEL_H) return fail(h, LSM_ERR_ARG, "lsm_solve_adjoint: not available for LSM_KERNEL_H");
    const void* bb[1] = {b};
    void* xx[1] = {x};
    return solve_batched(1, &h, bb, xx, iters, relres, nullptr, true);
}

extern "C" lsm_status lsm_set_contrast(lsm_t h, const double* dC, const double* drho) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_set_contrast: null handle");
    if (!dC || !drho) return fail(h, LSM_ERR_ARG, "lsm_set_contrast: null pointer argument");
    Store* s = h->s;
    const long long N = s->d.N;
    CK(h, cudaMemcpyAsync(s->dC64, dC, 21 * N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    CK(h, cudaMemcpyAsync(s->drho64, drho, N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    CK(h, launch_taper(s->d, s->taper, s->dC64, s->drho64, s->st, &h->nl));
    if (s->precision == LSM_MIXED) {
        CK(h, launch_d2f(s->dC64, s->dC32, 21 * N, s->st, &h->nl));
        CK(h, launch_d2f(s->drho64, s->drho32, N, s->st, &h->nl));
    }
    if (s->pair) {
        CK(h, launch_d2df(s->dC64, s->dCdf, 21 * N, s->st, &h->nl));
        CK(h, launch_d2df(s->drho64, s->drhodf, N, s->st, &h->nl));
    }
    return LSM_OK;
}

extern "C" lsm_status lsm_gradient(lsm_t h, const void* u, const void* lam, double* gC, double* grho, int accumulate) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_gradient: null handle");
    if (!u || !lam || !gC || !grho) return fail(h, LSM_ERR_ARG, "lsm_gradient: null pointer argument");
    Store* s = h->s;
    if (s->kernel == LSM_KERNEL_H) return fail(h, LSM_ERR_ARG, "lsm_gradient: not available for LSM_KERNEL_H");
    lsm_status rc = ensure_apply_ws(h);
    if (rc != LSM_OK) return rc;
    ApplySys<double> a;
    a.u = (const double2*)lam;
    a.out = nullptr;
    a.ghat = h->ghat64;
    a.w1 = s->w1_64;
    a.w2 = s->w2_64;
    a.omega2 = h->omega * h->omega;
    a.run = nullptr;
    a.count = nullptr;
    CK(h, cudaMemcpyAsync(s->a64, &a, sizeof(a), cudaMemcpyHostToDevice, s->st));
    Medium m = medium_of(s, 0);
    m.timer = nullptr;
    CK(h, launch_gradient(m, s->pl64, s->a64, (const double2*)u, gC, grho, accumulate, s->st, &h->nl));
    return LSM_OK;
}

extern "C" lsm_status lsm_source_gradient(lsm_t h, const double xs[3], const void* lam, double gM[6]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_source_gradient: null handle");
    if (!xs || !lam || !gM) return fail(h, LSM_ERR_ARG, "lsm_source_gradient: null pointer argument");
    Store* s = h->s;
    if (!s->grad_scratch) CK(h, cudaMalloc(&s->grad_scratch, (6 * 4096 + 8) * sizeof(double)));
    double* out = s->grad_scratch + 6 * 4096;
    CK(h, launch_source_gradient(s->d, s->lam, s->mu, s->rho, h->omega, s->green, xs, (const double2*)lam,
                                 s->grad_scratch, out, s->st, &h->nl));
    CK(h, cudaMemcpyAsync(gM, out, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(h, cudaStreamSynchronize(s->st));
    return LSM_OK;
}

// ---------------------------------------------------------------------------------------------
// FFT schedules and the tuner
// ---------------------------------------------------------------------------------------------
static bool schedule_ok(const int v[6]) {
    if (v[0] != 0 && v[0] != 1) return false;
    for (int k = 1; k < 6; ++k)
        if (v[k] < 0 || v[k] > (k == 3 ? 3 : 2)) return false;
    return true;
}

static lsm_status timer_events(lsm_t h) {
    KTimer& t = h->s->timer;
    if (t.ev) return LSM_OK;
    t.cap = 4096;
    t.ev = new cudaEvent_t[2 * t.cap];
    t.tag = new int[t.cap];
    for (int i = 0; i < 2 * t.cap; ++i) CK(h, cudaEventCreate(&t.ev[i]));
    return LSM_OK;
}

extern "C" lsm_status lsm_set_schedule(lsm_t h, int precision, const int v[6]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_set_schedule: null handle");
    if (!v || (precision != LSM_FP64 && precision != LSM_MIXED) || !schedule_ok(v))
        return fail(h, LSM_ERR_ARG, "lsm_set_schedule: invalid precision or variants");
    Store* s = h->s;
    CK(h, cudaStreamSynchronize(s->st));
    for (int k = 0; k < 6; ++k) s->sched[precision == LSM_MIXED ? 1 : 0][k] = v[k];
    drop_graphs(s->ws);   // captured iterations hold the old kernels
    return LSM_OK;
}

extern "C" lsm_status lsm_get_schedule(lsm_t h, int precision, int v[6]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_get_schedule: null handle");
    if (!v || (precision != LSM_FP64 && precision != LSM_MIXED))
        return fail(h, LSM_ERR_ARG, "lsm_get_schedule: invalid arguments");
    for (int k = 0; k < 6; ++k) v[k] = h->s->sched[precision == LSM_MIXED ? 1 : 0][k];
    return LSM_OK;
}

// declared with the solver workspace below
lsm_status tune_workspace(lsm_t h, int nsys);

// Times `reps` batched applies of nsys systems (one shared input, separate outputs and
// workspaces, the solver's layout) under each variant set and keeps the fastest variant per stage.
template <typename T>
static lsm_status tune_one(lsm_t h, int nsys, int reps, const void* u, void* out, int best[6]) {
    typedef typename cplx_of<T>::type C;
    Store* s = h->s;
    SolverWS& w = s->ws;
    KTimer& t = s->timer;
    const bool f32 = sizeof(T) == 4;
    const int p = f32 ? 1 : 0;
    std::vector<ApplySys<T>> a(nsys);
    for (int i = 0; i < nsys; ++i) {
        a[i].u = (const C*)u;
        a[i].out = (C*)((char*)out + (size_t)i * 3 * s->d.N * sizeof(C));
        a[i].ghat = f32 ? (const C*)h->ghat32 : (const C*)h->ghat64;
        const bool fp64_of_mixed = !f32 && s->precision == LSM_MIXED;
        a[i].w1 = fp64_of_mixed ? (C*)w.w1d[i] : (C*)w.w1[i];
        a[i].w2 = fp64_of_mixed ? (C*)w.w2d[i] : (C*)w.w2[i];
        a[i].omega2 = (T)(h->omega * h->omega);
        a[i].run = nullptr;
        a[i].count = nullptr;
    }
    ApplySys<T>* dev = (ApplySys<T>*)w.sys_x;
    CK(h, cudaMemcpyAsync(dev, a.data(), nsys * sizeof(ApplySys<T>), cudaMemcpyHostToDevice, s->st));
    const Plans& pl = f32 ? s->pl32 : s->pl64;
    // stage times (ms over `reps` batched applies) under the schedule currently set
    auto measure = [&](double (&ms)[6]) -> lsm_status {
        const Medium m = medium_of(s, f32);
        cudaError_t e = launch_apply<T>(m, pl, dev, nsys, s->st, &h->nl);   // warm-up
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "lsm_autotune");
        ktimer_flush(&t);
        double before[6];
        for (int k = 0; k < 6; ++k) before[k] = t.ms[6 * p + k];
        t.on = 1;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_apply<T>(m, pl, dev, nsys, s->st, &h->nl);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        t.on = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, "lsm_autotune");
        ktimer_flush(&t);
        for (int k = 0; k < 6; ++k) ms[k] = t.ms[6 * p + k] - before[k];
        return LSM_OK;
    };
    double best_ms[6];
    for (int k = 0; k < 6; ++k) {
        best[k] = 0;
        best_ms[k] = 1e300;
    }
    // stages 1..5: each variant set on all of them at once, the fastest kept per stage
    for (int var = 0; var <= 3; ++var) {
        s->sched[p][0] = 0;
        for (int k = 1; k < 6; ++k) s->sched[p][k] = (k == 3 || var < 3) ? var : 0;
        double ms[6];
        lsm_status rc = measure(ms);
        if (rc != LSM_OK) return rc;
        for (int k = 1; k < 6; ++k) {
            if (var == 3 && k != 3) continue;
            if (ms[k] < best_ms[k]) {
                best_ms[k] = ms[k];
                best[k] = var;
            }
        }
    }
    // stage 0 (separate stress and divergence, or fused): they also change what stage 1 times
    double two[2];
    for (int v0 = 0; v0 <= 1; ++v0) {
        for (int k = 1; k < 6; ++k) s->sched[p][k] = best[k];
        s->sched[p][0] = v0;
        double ms[6];
        lsm_status rc = measure(ms);
        if (rc != LSM_OK) return rc;
        two[v0] = ms[0] + ms[1];
    }
    best[0] = two[1] < two[0] ? 1 : 0;
    for (int k = 0; k < 6; ++k) s->sched[p][k] = best[k];
    return LSM_OK;
}

extern "C" lsm_status lsm_autotune(lsm_t h, int nsys, int reps, int v64[6], int v32[6]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_autotune: null handle");
    if (nsys < 1 || nsys > 64 || reps < 1 || reps > 100)
        return fail(h, LSM_ERR_ARG, "lsm_autotune: nsys must be in 1..64 and reps in 1..100");
    Store* s = h->s;
    lsm_status rc = tune_workspace(h, nsys);
    if (rc == LSM_OK) rc = timer_events(h);
    if (rc != LSM_OK) return rc;
    CK(h, cudaStreamSynchronize(s->st));
    KTimer& t = s->timer;
    const int was_on = t.on;
    t.on = 0;
    t.used = 0;
    t.open = 0;
    const size_t bytes = 3 * (size_t)s->d.N * sizeof(double2);
    void* buf = nullptr;
    CK(h, cudaMalloc(&buf, (1 + (size_t)nsys) * bytes));
    void* u = buf;
    void* out = (char*)buf + bytes;
    cudaError_t e = cudaMemsetAsync(u, 0, bytes, s->st);   // FFT time does not depend on the values
    int best64[6], best32[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) {
        rc = tune_one<double>(h, nsys, reps, u, out, best64);
        if (rc == LSM_OK && s->precision == LSM_MIXED) rc = tune_one<float>(h, nsys, reps, u, out, best32);
    }
    cudaStreamSynchronize(s->st);
    cudaFree(buf);
    t.on = was_on;
    t.used = 0;
    t.open = 0;
    for (int k = 0; k < 12; ++k) {
        t.ms[k] = 0.0;
        t.launches[k] = 0;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lsm_autotune");
    if (rc != LSM_OK) return rc;
    drop_graphs(s->ws);
    if (v64)
        for (int k = 0; k < 6; ++k) v64[k] = best64[k];
    if (v32)
        for (int k = 0; k < 6; ++k) v32[k] = best32[k];
    return LSM_OK;
}

extern "C" lsm_status lsm_dot_c64(lsm_t h, long long n, const void* a, const void* b, double out[2]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_dot_c64: null handle");
    if (!a || !b || !out || n < 0) return fail(h, LSM_ERR_ARG, "lsm_dot_c64: null pointer or negative length");
    Store* s = h->s;
    const int nblk = vec_blocks(n);
    double* scratch = nullptr;
    CK(h, cudaMalloc(&scratch, (2 * (size_t)nblk + 2) * sizeof(double)));
    cudaError_t e = launch_dot_c64((const float2*)a, (const float2*)b, n, scratch, nblk, scratch + 2 * nblk, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch + 2 * nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(h, e, "lsm_dot_c64");
    h->nl += 2;
    return LSM_OK;
}

extern "C" lsm_status lsm_timer_start(lsm_t h, int enable) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_timer_start: null handle");
    Store* s = h->s;
    CK(h, cudaStreamSynchronize(s->st));
    KTimer& t = s->timer;
    lsm_status rc = timer_events(h);
    if (rc != LSM_OK) return rc;
    t.on = enable ? 1 : 0;
    t.used = 0;
    t.open = 0;
    for (int i = 0; i < 12; ++i) {
        t.ms[i] = 0.0;
        t.launches[i] = 0;
    }
    CK(h, cudaMemsetAsync(s->counts, 0, 2 * sizeof(unsigned long long), s->st));
    CK(h, cudaStreamSynchronize(s->st));
    return LSM_OK;
}

extern "C" lsm_status lsm_timer_read(lsm_t h, double ms[12], long long launches[12], long long applies[2]) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_timer_read: null handle");
    Store* s = h->s;
    CK(h, cudaStreamSynchronize(s->st));
    ktimer_flush(&s->timer);
    unsigned long long c[2] = {0, 0};
    CK(h, cudaMemcpy(c, s->counts, sizeof(c), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 12; ++i) {
        if (ms) ms[i] = s->timer.ms[i];
        if (launches) launches[i] = s->timer.launches[i];
    }
    if (applies) {
        applies[0] = (long long)c[0];
        applies[1] = (long long)c[1];
    }
    return LSM_OK;
}

// ---------------------------------------------------------------------------------------------
// Operator apply without any device allocation.
//
// lsm_apply allocates its FP64 workspace with cudaMalloc on a handle's first apply.  Some callers
// cannot allocate at that point: a serving process whose device memory was reserved up front by
// another allocator (a framework's caching allocator holding the whole device), or a loop that must
// not stop on an out-of-memory error, or on cudaMalloc's implicit synchronisation, halfway through.
// lsm_apply_static gives them the same FP64 apply with its workspace taken from one library-wide
// array in device global memory (g_static_scratch, STATIC_SCRATCH_BYTES per device that loads the
// library, held until the process exits).
// ---------------------------------------------------------------------------------------------
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = 64ull << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_static_addr[MAX_DEVICES] = {nullptr};
std::mutex g_static_mu;

// Device address of g_static_scratch on device dev, which must be current; looked up once per
// device (the host-side symbol is only a stand-in and must never be handed to a kernel).
cudaError_t static_scratch_addr(int dev, void** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

// The argument block reaches the device as a kernel parameter (copied when the launch is made),
// so no host buffer has to outlive the call.
__global__ void k_put_apply_args(ApplySys<double>* dst, ApplySys<double> a) { *dst = a; }

// bytes of the static array one apply with the handle's geometry uses: the argument block and the
// two workspaces the apply itself sizes with apply_ws_elems
size_t static_apply_bytes(const Store* s, long long* e1, long long* e2) {
    apply_ws_elems(s->d, s->kernel, e1, e2);
    return align_up(sizeof(ApplySys<double>)) + align_up(*e1 * sizeof(double2)) + align_up(*e2 * sizeof(double2));
}

}  // namespace

extern "C" lsm_status lsm_apply_static(lsm_t h, const void* u, void* Au) {
    if (!h) return fail(nullptr, LSM_ERR_ARG, "lsm_apply_static: null handle");
    if (!u || !Au || u == Au) return fail(h, LSM_ERR_ARG, "lsm_apply_static: u and Au must be distinct non-null device buffers");
    Store* s = h->s;
    if (s->kernel == LSM_KERNEL_H) return fail(h, LSM_ERR_ARG, "lsm_apply_static: not available for LSM_KERNEL_H");
    int cur = -1;
    CK(h, cudaGetDevice(&cur));
    if (cur != s->device)
        return fail(h, LSM_ERR_ARG, "lsm_apply_static: the handle's device must be the current device");
    long long e1, e2;
    const size_t need = static_apply_bytes(s, &e1, &e2);
    if (need > STATIC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg), "lsm_apply_static: grid %dx%dx%d needs %zu bytes of scratch, more than the %zu-byte static array",
                 s->d.nx, s->d.ny, s->d.nz, need, (size_t)STATIC_SCRATCH_BYTES);
        return fail(h, LSM_ERR_ARG, msg);
    }
    void* base = nullptr;
    CK(h, static_scratch_addr(cur, &base));
    char* p = (char*)base;
    ApplySys<double>* dev_args = (ApplySys<double>*)p;
    double2* w1 = (double2*)(p + align_up(sizeof(ApplySys<double>)));
    double2* w2 = (double2*)((char*)w1 + align_up(e1 * sizeof(double2)));
    // every workspace element the apply reads is written earlier in the same apply, so nothing
    // in the array has to start at zero
    ApplySys<double> a;
    a.u = (const double2*)u;
    a.out = (double2*)Au;
    a.ghat = h->ghat64;
    a.w1 = w1;
    a.w2 = w2;
    a.omega2 = h->omega * h->omega;
    a.run = nullptr;
    a.count = nullptr;
    k_put_apply_args<<<1, 1, 0, s->st>>>(dev_args, a);
    CK(h, cudaGetLastError());
    h->nl += 1;
    Medium m = medium_of(s, 0);
    m.timer = nullptr;
    cudaError_t e = launch_apply<double>(m, s->pl64, dev_args, 1, s->st, &h->nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "lsm_apply_static");
    return LSM_OK;
}

extern "C" lsm_status lsm_time_traces(int nf, double df, int ntr, const void* spectra, int nt, double dt, double fp,
                                      double t0, double* traces, void* stream) {
    if (nf < 1 || nf > 12288 || ntr < 1 || nt < 1 || !spectra || !traces || !(df > 0) || !(dt > 0) || !(fp > 0) ||
        !std::isfinite(t0))
        return fail(nullptr, LSM_ERR_ARG, "lsm_time_traces: need 1 <= nf <= 12288, ntr, nt >= 1, df, dt, fp > 0");
    cudaError_t e = launch_time_traces(nf, df, ntr, (const double2*)spectra, nt, dt, fp, t0, traces, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lsm_time_traces");
    return LSM_OK;
}

// Seismogram chain (Sec. 4.1.2): LS solves at f_k = k df wave by wave, receiver gather, traces.
extern "C" lsm_status lsm_seismograms(lsm_t base, int nf, double df, const double M[6], const double xs[3], int nrec,
                                      const int* rec, int nt, double dt, double fp, double t0, double* traces, int wave,
                                      int* iters, double* relres) {
    if (!base) return fail(nullptr, LSM_ERR_ARG, "lsm_seismograms: null handle");
    if (nf < 2 || nf > 12288 || !(df > 0) || !std::isfinite(df) || !M || !xs || nrec < 1 || nrec > (1 << 20) || !rec ||
        nt < 1 || !(dt > 0) || !(fp > 0) || !std::isfinite(t0) || !traces || wave < 1 || wave > 256)
        return fail(base, LSM_ERR_ARG,
                    "lsm_seismograms: need 2 <= nf <= 12288, df, dt, fp > 0, 1 <= nrec, nt >= 1, 1 <= wave <= 256 and "
                    "non-null pointers");
    Store* s = base->s;
    const Dims& d = s->d;
    std::vector<long long> node(nrec);
    for (int r = 0; r < nrec; ++r) {
        const int ix = rec[3 * r], iy = rec[3 * r + 1], iz = rec[3 * r + 2];
        if (ix < 0 || ix >= d.nx || iy < 0 || iy >= d.ny || iz < 0 || iz >= d.nz)
            return fail(base, LSM_ERR_ARG, "lsm_seismograms: receiver node outside the grid");
        node[r] = ((long long)iz * d.ny + iy) * d.nx + ix;
    }
    const cudaStream_t st = s->st;
    const long long ntr = 3LL * nrec;
    long long* d_node = nullptr;
    double2* d_U = nullptr;
    CK(base, cudaMalloc(&d_node, nrec * sizeof(long long)));
    cudaError_t e = cudaMalloc(&d_U, (size_t)nf * ntr * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_node, node.data(), nrec * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_U, 0, (size_t)nf * ntr * sizeof(double2), st);
    lsm_status rc = e == cudaSuccess ? LSM_OK : cuda_fail(base, e, "lsm_seismograms: receiver buffers");
    bool on_node = false;
    if (iters) iters[0] = 0;
    if (relres) relres[0] = 0.0;
    const size_t fbytes = 3 * (size_t)d.N * sizeof(double2);
    for (int k0 = 1; k0 < nf && rc == LSM_OK; k0 += wave) {
        const int m = (nf - k0 < wave) ? nf - k0 : wave;
        std::vector<lsm_t> hs(m, nullptr);
        std::vector<void*> bs(m, nullptr), xv(m, nullptr);
        std::vector<int> it(m, 0);
        std::vector<double> rr(m, 0.0);
        for (int j = 0; j < m && rc == LSM_OK; ++j) {
            rc = lsm_create_shared(&hs[j], base, 2.0 * M_PI * (k0 + j) * df);
            if (rc != LSM_OK) {
                base->err = std::string("lsm_seismograms: ") + g_err;
                break;
            }
            e = cudaMalloc(&bs[j], fbytes);
            if (e == cudaSuccess) e = cudaMalloc(&xv[j], fbytes);
            if (e != cudaSuccess) {
                rc = cuda_fail(base, e, "lsm_seismograms: fields");
                break;
            }
            const lsm_status r0 = lsm_source(hs[j], M, xs, bs[j]);
            if (r0 == LSM_WARN_SOURCE_ON_NODE) on_node = true;
            else if (r0 != LSM_OK) {
                base->err = hs[j]->err;
                rc = r0;
                break;
            }
            e = cudaMemsetAsync(xv[j], 0, fbytes, st);
            if (e != cudaSuccess) rc = cuda_fail(base, e, "lsm_seismograms: initial guess");
        }
        if (rc == LSM_OK) {
            rc = lsm_solve_batched(m, hs.data(), bs.data(), xv.data(), it.data(), rr.data(), nullptr);
            if (rc != LSM_OK) base->err = "lsm_seismograms: " + hs[0]->err;
        }
        for (int j = 0; j < m && rc == LSM_OK; ++j) {
            e = launch_gather_receivers((const double2*)xv[j], d.N, d_node, nrec, d_U + (size_t)(k0 + j) * ntr, st);
            if (e != cudaSuccess) rc = cuda_fail(base, e, "lsm_seismograms: receiver gather");
            base->nl += 1;
            if (iters) iters[k0 + j] = it[j];
            if (relres) relres[k0 + j] = rr[j];
        }
        cudaStreamSynchronize(st);
        for (int j = 0; j < m; ++j) {
            cudaFree(bs[j]);
            cudaFree(xv[j]);
            if (hs[j]) {
                base->nl += hs[j]->nl;
                lsm_destroy(hs[j]);
            }
        }
    }
    if (rc == LSM_OK) {
        e = launch_time_traces(nf, df, (int)ntr, d_U, nt, dt, fp, t0, traces, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(base, e, "lsm_seismograms: time traces");
        base->nl += 1;
    }
    cudaStreamSynchronize(st);
    cudaFree(d_node);
    cudaFree(d_U);
    if (rc == LSM_OK && on_node) {
        base->err = "lsm_seismograms: a grid node coincides with the source; u0 set to 0 there";
        return LSM_WARN_SOURCE_ON_NODE;
    }
    return rc;
}
