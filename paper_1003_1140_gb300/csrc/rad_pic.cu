// rad_pic.cu -- the small live 2D3V PIC of the two-stream setup (Sec. 2.1)
// that drives the radiation diagnostic in situ (C ABI in include/rad_pic.h).
//
// One step (state x^n, u^{n-1/2}, E^n, B^n):
//   1. push_deposit: one thread per particle gathers E^n, B^n from the
//      staggered Yee points with linear weights, Boris-pushes u to n+1/2,
//      moves x to n+1 and deposits the charge-conserving current of the move
//      (Esirkepov's decomposition for linear shapes on the 4 x 4 node stencil
//      the old and new positions share) with FP64 atomics, then wraps x;
//   2. faraday: B^{n+1/2} = B^n - dt/2 curl E^n;
//   3. ampere:  E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2});
//   4. faraday: B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}.
// FP64 throughout (the diagnostic's FP64 parity chain reaches back into the
// particle state); a PIC step costs a few hundred FP64 operations per
// particle, which this GPU's FP64 pipe (1/64 of FP32) sustains at a few
// hundred million particles per second -- far below the diagnostic's rate,
// so the tracked subset, not the push, sets the in-situ cost.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "rad.h"
#include "rad_internal.cuh"
#include "rad_pic.h"

namespace {

constexpr int kMaxSpecies = 8;

struct PicDev {
    int n;
    double d, inv_d, dt, L;
    const double* E;   // [3][n][n]
    const double* B;
    double* J;
    double* x;         // [3][N]
    double* u;
    int64_t N;
    int n_species;
    int64_t off[kMaxSpecies + 1];
    double qm[kMaxSpecies];   // q / m
    double qw[kMaxSpecies];   // q w (macro charge)
};

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Linear interpolation of a field stored at (j + oy, k + oz) (offsets 0 or 1/2
// folded into the coordinates by the caller).
__device__ __forceinline__ double interp(const double* F, int n, int j, double fy, int k, double fz)
{
    const int j0 = wrap(j, n), j1 = wrap(j + 1, n), k0 = wrap(k, n), k1 = wrap(k + 1, n);
    return (1.0 - fy) * (1.0 - fz) * F[j0 * n + k0] + fy * (1.0 - fz) * F[j1 * n + k0] +
           (1.0 - fy) * fz * F[j0 * n + k1] + fy * fz * F[j1 * n + k1];
}

// CIC weights of s (cell units) on nodes base .. base + 3.
__device__ __forceinline__ void node_weights(double s, int base, double (&W)[4])
{
    const double fl = floor(s);
    const int i = (int)fl - base;
    const double f = s - fl;
#pragma unroll
    for (int c = 0; c < 4; ++c) W[c] = (c == i ? 1.0 - f : 0.0) + (c == i + 1 ? f : 0.0);
}

__device__ __forceinline__ void add(double* a, double v)
{
    if (v != 0.0) atomicAdd(a, v);
}

__global__ void __launch_bounds__(256) push_deposit(const PicDev p)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int sp = 0;
    while (sp + 1 < p.n_species && i >= p.off[sp + 1]) ++sp;
    const int n = p.n;
    const int64_t N = p.N;
    const int64_t nn = (int64_t)n * n;
    double x0 = p.x[i], y0 = p.x[N + i], z0 = p.x[2 * N + i];
    double u0 = p.u[i], u1 = p.u[N + i], u2 = p.u[2 * N + i];

    // ---- gather E^n, B^n at (y0, z0)
    const double sy = y0 * p.inv_d, sz = z0 * p.inv_d;
    const double jnf = floor(sy), jhf = floor(sy - 0.5), knf = floor(sz), khf = floor(sz - 0.5);
    const int jn = (int)jnf, jh = (int)jhf, kn = (int)knf, kh = (int)khf;
    const double fyn = sy - jnf, fyh = (sy - 0.5) - jhf, fzn = sz - knf, fzh = (sz - 0.5) - khf;
    const double Ex = interp(p.E, n, jn, fyn, kn, fzn);
    const double Ey = interp(p.E + nn, n, jh, fyh, kn, fzn);
    const double Ez = interp(p.E + 2 * nn, n, jn, fyn, kh, fzh);
    const double Bx = interp(p.B, n, jh, fyh, kh, fzh);
    const double By = interp(p.B + nn, n, jn, fyn, kh, fzh);
    const double Bz = interp(p.B + 2 * nn, n, jh, fyh, kn, fzn);

    // ---- relativistic Boris
    const double h = 0.5 * p.qm[sp] * p.dt;
    const double m0 = u0 + h * Ex, m1 = u1 + h * Ey, m2 = u2 + h * Ez;
    const double gm = sqrt(1.0 + (m0 * m0 + m1 * m1 + m2 * m2));
    const double t0 = h / gm * Bx, t1 = h / gm * By, t2 = h / gm * Bz;
    const double tt = 2.0 / (1.0 + (t0 * t0 + t1 * t1 + t2 * t2));
    const double s0 = tt * t0, s1 = tt * t1, s2 = tt * t2;
    const double p0 = m0 + (m1 * t2 - m2 * t1), p1 = m1 + (m2 * t0 - m0 * t2), p2 = m2 + (m0 * t1 - m1 * t0);
    const double q0 = m0 + (p1 * s2 - p2 * s1), q1 = m1 + (p2 * s0 - p0 * s2), q2 = m2 + (p0 * s1 - p1 * s0);
    u0 = q0 + h * Ex;
    u1 = q1 + h * Ey;
    u2 = q2 + h * Ez;
    const double g = sqrt(1.0 + (u0 * u0 + u1 * u1 + u2 * u2));
    const double v0 = u0 / g, v1 = u1 / g, v2 = u2 / g;
    const double x1 = x0 + p.dt * v0, y1 = y0 + p.dt * v1, z1 = z0 + p.dt * v2;

    // ---- charge-conserving current of the move (y0, z0) -> (y1, z1)
    {
        const double s0y = y0 * p.inv_d, s0z = z0 * p.inv_d;
        const double s1y = y1 * p.inv_d, s1z = z1 * p.inv_d;
        const int by = (int)floor(s0y) - 1, bz = (int)floor(s0z) - 1;
        double S0y[4], S1y[4], S0z[4], S1z[4];
        node_weights(s0y, by, S0y);
        node_weights(s1y, by, S1y);
        node_weights(s0z, bz, S0z);
        node_weights(s1z, bz, S1z);
        const double qw = p.qw[sp];
        const double cx = qw * v0 / (p.d * p.d), cyz = -qw / (p.d * p.dt);
        double cy_run[4] = {0.0, 0.0, 0.0, 0.0};   // running sum over a, per b
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double dSy = S1y[a] - S0y[a];
            const int j = wrap(by + a, n);
            double cz_run = 0.0;                   // running sum over b for this a
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const double dSz = S1z[b] - S0z[b];
                const int k = wrap(bz + b, n);
                const double Wx = S0y[a] * S0z[b] + 0.5 * dSy * S0z[b] + 0.5 * S0y[a] * dSz +
                                  dSy * dSz / 3.0;
                cy_run[b] += dSy * (S0z[b] + S1z[b]) * 0.5;
                cz_run += (S0y[a] + S1y[a]) * dSz * 0.5;
                double* Jc = p.J + (int64_t)j * n + k;
                add(Jc, cx * Wx);
                add(Jc + nn, cyz * cy_run[b]);
                add(Jc + 2 * nn, cyz * cz_run);
            }
        }
    }

    // ---- wrap into [0, L) and store
    auto wrapL = [&](double c) { return c < 0.0 ? c + p.L : (c >= p.L ? c - p.L : c); };
    p.x[i] = wrapL(x1);
    p.x[N + i] = wrapL(y1);
    p.x[2 * N + i] = wrapL(z1);
    p.u[i] = u0;
    p.u[N + i] = u1;
    p.u[2 * N + i] = u2;
}

// B -= c curl E (c = dt/2), on the B points; d/dx = 0.
__global__ void faraday(const double* __restrict__ E, double* __restrict__ B, int n, double inv_d,
                        double c)
{
    const int64_t nn = (int64_t)n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / n), k = (int)(q % n);
        const int jp = j + 1 == n ? 0 : j + 1, kp = k + 1 == n ? 0 : k + 1;
        const double* Ex = E;
        const double* Ey = E + nn;
        const double* Ez = E + 2 * nn;
        const double cx = (Ez[(int64_t)jp * n + k] - Ez[q]) * inv_d - (Ey[(int64_t)j * n + kp] - Ey[q]) * inv_d;
        const double cy = (Ex[(int64_t)j * n + kp] - Ex[q]) * inv_d;
        const double cz = -(Ex[(int64_t)jp * n + k] - Ex[q]) * inv_d;
        B[q] -= c * cx;
        B[nn + q] -= c * cy;
        B[2 * nn + q] -= c * cz;
    }
}

// E += dt (curl B - J), on the E points; d/dx = 0.
__global__ void ampere(double* __restrict__ E, const double* __restrict__ B,
                       const double* __restrict__ J, int n, double inv_d, double dt)
{
    const int64_t nn = (int64_t)n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / n), k = (int)(q % n);
        const int jm = j == 0 ? n - 1 : j - 1, km = k == 0 ? n - 1 : k - 1;
        const double* Bx = B;
        const double* By = B + nn;
        const double* Bz = B + 2 * nn;
        const double cx = (Bz[q] - Bz[(int64_t)jm * n + k]) * inv_d - (By[q] - By[(int64_t)j * n + km]) * inv_d;
        const double cy = (Bx[q] - Bx[(int64_t)j * n + km]) * inv_d;
        const double cz = -(Bx[q] - Bx[(int64_t)jm * n + k]) * inv_d;
        E[q] += dt * (cx - J[q]);
        E[nn + q] += dt * (cy - J[nn + q]);
        E[2 * nn + q] += dt * (cz - J[2 * nn + q]);
    }
}

// Positions into [0, L) (init: the kernels' index arithmetic relies on it; the
// push keeps it, moving particles by under one cell per step).
__global__ void wrap_positions(double* x, int64_t n3, double L)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        double w = v - L * floor(v / L);
        if (!(w >= 0.0 && w < L)) w = 0.0;    // non-finite input, or rounding up to L
        x[i] = w;
    }
}

__global__ void gather_range(const double* __restrict__ x, const double* __restrict__ u, int64_t N,
                             int64_t first, int64_t count, double* __restrict__ xo,
                             double* __restrict__ uo)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xo[c * count + i] = x[c * N + first + i];
            uo[c * count + i] = u[c * N + first + i];
        }
    }
}

// out[0] += sum (E^2 + B^2)/2 d^2, out[1] += sum w m (gamma - 1)
__global__ void energy_kernel(const PicDev p, const double* __restrict__ mw, double* out)
{
    const int64_t nn = (int64_t)p.n * p.n;
    double ef = 0.0, ek = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * nn;
         q += (int64_t)gridDim.x * blockDim.x)
        ef += 0.5 * (p.E[q] * p.E[q] + p.B[q] * p.B[q]) * p.d * p.d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int sp = 0;
        while (sp + 1 < p.n_species && i >= p.off[sp + 1]) ++sp;
        const double a = p.u[i], b = p.u[p.N + i], c = p.u[2 * p.N + i];
        ek += mw[sp] * (sqrt(1.0 + (a * a + b * b + c * c)) - 1.0);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ef += __shfl_down_sync(0xffffffffu, ef, o);
        ek += __shfl_down_sync(0xffffffffu, ek, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, ef);
        atomicAdd(out + 1, ek);
    }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

bool is_dev(const void* ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct rad_pic {
    PicDev dev{};
    double* E = nullptr;
    double* B = nullptr;
    double* J = nullptr;
    double* x = nullptr;
    double* u = nullptr;
    double* mw = nullptr;       // per-species m w (device)
    double* en = nullptr;       // energy accumulators (device)
    double* xt = nullptr;       // staging for the tracked particles
    double* ut = nullptr;
    int64_t staged = 0;
    int64_t steps = 0;
    cudaEvent_t staged_ev = nullptr;   // staging buffers written (PIC stream)
    cudaEvent_t read_ev = nullptr;     // staging buffers read (radiation stream)
    cudaStream_t st = nullptr;
    std::string err;
};

static int pfail(rad_pic* p, int rc, const std::string& what, cudaError_t e = cudaSuccess)
{
    if (p) p->err = e != cudaSuccess ? what + ": " + cudaGetErrorString(e) : what;
    return rc;
}

#define PCU(call)                                                        \
    do {                                                                 \
        const cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return pfail(p, RAD_PIC_ECUDA, #call, e_); \
    } while (0)

static int pic_step(rad_pic* p)
{
    const int64_t nn = (int64_t)p->dev.n * p->dev.n;
    PCU(cudaMemsetAsync(p->J, 0, 3 * nn * sizeof(double), p->st));
    if (p->dev.N > 0) push_deposit<<<(unsigned)((p->dev.N + 255) / 256), 256, 0, p->st>>>(p->dev);
    PCU(cudaGetLastError());
    const double inv_d = p->dev.inv_d, dt = p->dev.dt;
    faraday<<<grid_for(nn), 256, 0, p->st>>>(p->E, p->B, p->dev.n, inv_d, 0.5 * dt);
    ampere<<<grid_for(nn), 256, 0, p->st>>>(p->E, p->B, p->J, p->dev.n, inv_d, dt);
    faraday<<<grid_for(nn), 256, 0, p->st>>>(p->E, p->B, p->dev.n, inv_d, 0.5 * dt);
    PCU(cudaGetLastError());
    ++p->steps;
    return RAD_PIC_OK;
}

extern "C" {

int rad_pic_init(rad_pic** out, int32_t n, double d, double dt, const rad_pic_species* sp,
                 int32_t n_species, const double* x, const double* u, void* cuda_stream)
{
    if (!out) return RAD_PIC_EINVAL;
    *out = nullptr;
    if (n < 4 || n > 16384 || !(d > 0.0) || !(dt > 0.0) || !std::isfinite(d) ||
        !std::isfinite(dt) || !(dt < d / std::sqrt(2.0)) ||
        n_species < 0 || n_species > kMaxSpecies || (n_species > 0 && !sp))
        return RAD_PIC_EINVAL;
    int64_t N = 0;
    for (int s = 0; s < n_species; ++s) {
        if (sp[s].count < 0 || !(sp[s].mass > 0.0) || !std::isfinite(sp[s].charge) ||
            !std::isfinite(sp[s].weight))
            return RAD_PIC_EINVAL;
        N += sp[s].count;
    }
    if (N > 0 && (!x || !u)) return RAD_PIC_EINVAL;
    rad_pic* p = new (std::nothrow) rad_pic();
    if (!p) return RAD_PIC_ENOMEM;
    p->st = (cudaStream_t)cuda_stream;
    const int64_t nn = (int64_t)n * n;
    auto bail = [&](int rc) {
        rad_pic_destroy(p);
        return rc;
    };
#define PMAL(ptr, bytes)                                                              \
    do {                                                                              \
        if (cudaMalloc(&(ptr), (bytes) > 0 ? (bytes) : 8) != cudaSuccess) {           \
            cudaGetLastError();                                                       \
            return bail(RAD_PIC_ENOMEM);                                              \
        }                                                                             \
    } while (0)
    PMAL(p->E, 3 * nn * sizeof(double));
    PMAL(p->B, 3 * nn * sizeof(double));
    PMAL(p->J, 3 * nn * sizeof(double));
    PMAL(p->x, 3 * N * sizeof(double));
    PMAL(p->u, 3 * N * sizeof(double));
    PMAL(p->mw, kMaxSpecies * sizeof(double));
    PMAL(p->en, 2 * sizeof(double));
#undef PMAL
    if (cudaMemset(p->E, 0, 3 * nn * sizeof(double)) != cudaSuccess ||
        cudaMemset(p->B, 0, 3 * nn * sizeof(double)) != cudaSuccess ||
        (N > 0 && (cudaMemcpy(p->x, x, 3 * N * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
                   cudaMemcpy(p->u, u, 3 * N * sizeof(double), cudaMemcpyDefault) != cudaSuccess)))
        return bail(RAD_PIC_ECUDA);
    PicDev& D = p->dev;
    D.n = n;
    D.d = d;
    D.inv_d = 1.0 / d;
    D.dt = dt;
    D.L = n * d;
    D.E = p->E;
    D.B = p->B;
    D.J = p->J;
    D.x = p->x;
    D.u = p->u;
    D.N = N;
    D.n_species = n_species;
    double mw[kMaxSpecies] = {0};
    D.off[0] = 0;
    for (int s = 0; s < n_species; ++s) {
        D.off[s + 1] = D.off[s] + sp[s].count;
        D.qm[s] = sp[s].charge / sp[s].mass;
        D.qw[s] = sp[s].charge * sp[s].weight;
        mw[s] = sp[s].mass * sp[s].weight;
    }
    if (cudaMemcpy(p->mw, mw, sizeof mw, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(RAD_PIC_ECUDA);
    if (N > 0) {
        wrap_positions<<<grid_for(3 * N), 256>>>(p->x, 3 * N, D.L);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
            return bail(RAD_PIC_ECUDA);
    }
    *out = p;
    return RAD_PIC_OK;
}

int rad_pic_set_fields(rad_pic* p, const double* E, const double* B)
{
    if (!p) return RAD_PIC_EINVAL;
    const size_t bytes = 3 * (size_t)p->dev.n * p->dev.n * sizeof(double);
    if (E) PCU(cudaMemcpyAsync(p->E, E, bytes, cudaMemcpyDefault, p->st));
    if (B) PCU(cudaMemcpyAsync(p->B, B, bytes, cudaMemcpyDefault, p->st));
    PCU(cudaStreamSynchronize(p->st));
    return RAD_PIC_OK;
}

int rad_pic_get_fields(rad_pic* p, double* E, double* B)
{
    if (!p) return RAD_PIC_EINVAL;
    const size_t bytes = 3 * (size_t)p->dev.n * p->dev.n * sizeof(double);
    if (E) PCU(cudaMemcpyAsync(E, p->E, bytes, cudaMemcpyDefault, p->st));
    if (B) PCU(cudaMemcpyAsync(B, p->B, bytes, cudaMemcpyDefault, p->st));
    PCU(cudaStreamSynchronize(p->st));
    return RAD_PIC_OK;
}

int rad_pic_get_particles(rad_pic* p, double* x, double* u)
{
    if (!p) return RAD_PIC_EINVAL;
    const size_t bytes = 3 * (size_t)p->dev.N * sizeof(double);
    if (x && bytes) PCU(cudaMemcpyAsync(x, p->x, bytes, cudaMemcpyDefault, p->st));
    if (u && bytes) PCU(cudaMemcpyAsync(u, p->u, bytes, cudaMemcpyDefault, p->st));
    PCU(cudaStreamSynchronize(p->st));
    return RAD_PIC_OK;
}

int rad_pic_step(rad_pic* p, int32_t n_steps)
{
    if (!p || n_steps < 0) return pfail(p, RAD_PIC_EINVAL, "rad_pic_step: bad arguments");
    for (int32_t s = 0; s < n_steps; ++s) {
        const int rc = pic_step(p);
        if (rc) return rc;
    }
    return RAD_PIC_OK;
}

int64_t rad_pic_steps_done(const rad_pic* p) { return p ? p->steps : -1; }

int rad_pic_tracked(rad_pic* p, int64_t first, int64_t count, double* x_out, double* u_out)
{
    if (!p || first < 0 || count < 0 || first + count > p->dev.N || !x_out || !u_out ||
        !is_dev(x_out) || !is_dev(u_out))
        return pfail(p, RAD_PIC_EINVAL, "rad_pic_tracked: range or device buffers");
    if (count == 0) return RAD_PIC_OK;
    gather_range<<<grid_for(count), 256, 0, p->st>>>(p->x, p->u, p->dev.N, first, count, x_out, u_out);
    PCU(cudaGetLastError());
    return RAD_PIC_OK;
}

int rad_pic_run_coupled(rad_pic* p, rad_ctx* r, int64_t first, int64_t count, int32_t n_steps)
{
    if (!p || !r || n_steps < 0 || first < 0 || count < 1 || first + count > p->dev.N)
        return pfail(p, RAD_PIC_EINVAL, "rad_pic_run_coupled: bad arguments");
    if (rad::ctx_particles(r) != count)
        return pfail(p, RAD_PIC_EINVAL, "rad_pic_run_coupled: count differs from the radiation "
                                        "context's particle count");
    if (p->staged < count) {
        if (p->xt) cudaFree(p->xt);
        if (p->ut) cudaFree(p->ut);
        p->xt = p->ut = nullptr;
        p->staged = 0;
        if (cudaMalloc(&p->xt, 3 * count * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->ut, 3 * count * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return pfail(p, RAD_PIC_ENOMEM, "rad_pic_run_coupled: staging buffers");
        }
        p->staged = count;
    }
    if (!p->staged_ev) {
        PCU(cudaEventCreateWithFlags(&p->staged_ev, cudaEventDisableTiming));
        PCU(cudaEventCreateWithFlags(&p->read_ev, cudaEventDisableTiming));
    }
    // the radiation context may order its work on another stream: its reads of
    // the staging buffers wait for the gather, and the next gather waits for
    // those reads
    const cudaStream_t rs = rad::ctx_stream(r);
    const bool other = rs != p->st;
    auto hand_over = [&]() -> int {
        // a state the context has already received (the final state of a previous run)
        if (rad::ctx_next_step(r) == p->steps + 1) return RAD_PIC_OK;
        if (other) PCU(cudaStreamWaitEvent(p->st, p->read_ev, 0));
        gather_range<<<grid_for(count), 256, 0, p->st>>>(p->x, p->u, p->dev.N, first, count, p->xt,
                                                         p->ut);
        PCU(cudaGetLastError());
        if (other) {
            PCU(cudaEventRecord(p->staged_ev, p->st));
            PCU(cudaStreamWaitEvent(rs, p->staged_ev, 0));
        }
        const int rc = rad_accumulate(r, p->steps, p->xt, p->ut);
        if (rc != RAD_OK) return pfail(p, RAD_PIC_ERAD, std::string("rad_accumulate: ") + rad_last_error(r));
        if (other) PCU(cudaEventRecord(p->read_ev, rs));
        return RAD_PIC_OK;
    };
    for (int32_t s = 0; s < n_steps; ++s) {
        int rc = hand_over();
        if (rc) return rc;
        rc = pic_step(p);
        if (rc) return rc;
    }
    return hand_over();
}

int rad_pic_energy(rad_pic* p, double* field, double* kinetic)
{
    if (!p) return RAD_PIC_EINVAL;
    PCU(cudaMemsetAsync(p->en, 0, 2 * sizeof(double), p->st));
    energy_kernel<<<grid_for(std::max<int64_t>(p->dev.N, 3 * (int64_t)p->dev.n * p->dev.n)), 256, 0,
                    p->st>>>(p->dev, p->mw, p->en);
    PCU(cudaGetLastError());
    double h[2];
    PCU(cudaMemcpyAsync(h, p->en, sizeof h, cudaMemcpyDeviceToHost, p->st));
    PCU(cudaStreamSynchronize(p->st));
    if (field) *field = h[0];
    if (kinetic) *kinetic = h[1];
    return RAD_PIC_OK;
}

const char* rad_pic_last_error(const rad_pic* p) { return p ? p->err.c_str() : "null context"; }

void rad_pic_destroy(rad_pic* p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    for (double* q : {p->E, p->B, p->J, p->x, p->u, p->mw, p->en, p->xt, p->ut})
        if (q) cudaFree(q);
    if (p->staged_ev) cudaEventDestroy(p->staged_ev);
    if (p->read_ev) cudaEventDestroy(p->read_ev);
    delete p;
}

}  // extern "C"
