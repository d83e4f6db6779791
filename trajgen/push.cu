// push.cu -- GPU Boris pusher of the synthetic-trajectory generator.
//
// Input generation only (none of the radiation method's arithmetic): the
// same static mode field and Boris steps as trajgen.boris_push, in FP32
// arithmetic, for workloads too large to push with NumPy.  State and outputs
// are FP64 arrays holding FP32-representable values.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kMaxModes = 128;

__global__ void boris_kernel(int64_t N, int64_t n_calls, float L, float dt, const double* qm,
                             int n_modes, const double* ky, const double* kz, const double* psi,
                             const double* amp, double* xs, double* us, double* X, double* U)
{
    __shared__ float sky[kMaxModes], skz[kMaxModes], spsi[kMaxModes], samp[kMaxModes];
    for (int i = threadIdx.x; i < n_modes; i += blockDim.x) {
        sky[i] = (float)ky[i];
        skz[i] = (float)kz[i];
        spsi[i] = (float)psi[i];
        samp[i] = (float)amp[i];
    }
    __syncthreads();
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    float x0 = (float)xs[j], x1 = (float)xs[N + j], x2 = (float)xs[2 * N + j];
    float u0 = (float)us[j], u1 = (float)us[N + j], u2 = (float)us[2 * N + j];
    const float q = (float)qm[j];
    for (int64_t c = 0; c < n_calls; ++c) {
        double* Xc = X + c * 3 * N;
        double* Uc = U + c * 3 * N;
        Xc[j] = x0;
        Xc[N + j] = x1;
        Xc[2 * N + j] = x2;
        Uc[j] = u0;
        Uc[N + j] = u1;
        Uc[2 * N + j] = u2;
        // B = (0, dA/dz, -dA/dy), A = sum a cos(ky y + kz z + psi)
        float By = 0.f, Bz = 0.f;
        for (int i = 0; i < n_modes; ++i) {
            const float s = samp[i] * sinf(sky[i] * x1 + skz[i] * x2 + spsi[i]);
            By -= s * skz[i];
            Bz += s * sky[i];
        }
        float g = sqrtf(1.f + u0 * u0 + u1 * u1 + u2 * u2);
        const float f = 0.5f * dt * q / g;
        const float t1 = f * By, t2 = f * Bz;
        const float tt = t1 * t1 + t2 * t2;
        const float s1 = 2.f * t1 / (1.f + tt), s2 = 2.f * t2 / (1.f + tt);
        // u' = u + u x t, t = (0, t1, t2)
        const float p0 = u0 + (u1 * t2 - u2 * t1);
        const float p1 = u1 + (-u0 * t2);
        const float p2 = u2 + (u0 * t1);
        // u+ = u + u' x s, s = (0, s1, s2)
        u0 = u0 + (p1 * s2 - p2 * s1);
        u1 = u1 + (-p0 * s2);
        u2 = u2 + (p0 * s1);
        g = sqrtf(1.f + u0 * u0 + u1 * u1 + u2 * u2);
        x0 += dt * u0 / g;
        x1 += dt * u1 / g;
        x2 += dt * u2 / g;
        x0 -= L * floorf(x0 / L);
        x1 -= L * floorf(x1 / L);
        x2 -= L * floorf(x2 / L);
    }
    xs[j] = x0;
    xs[N + j] = x1;
    xs[2 * N + j] = x2;
    us[j] = u0;
    us[N + j] = u1;
    us[2 * N + j] = u2;
}

}  // namespace

extern "C" {

// Write n_calls consecutive leapfrog states (x_s, u_{s-1/2}) of N particles
// to X, U ([n_calls][3][N], device) and advance the state xs, us ([3][N],
// device) past them.  qm: [N] charge/mass; modes: [n_modes] device arrays.
// Returns 0, 1 on bad arguments, 2 on a CUDA error.
int tg_push(int64_t N, int64_t n_calls, double L, double dt, const double* qm, int n_modes,
            const double* ky, const double* kz, const double* psi, const double* amp,
            double* xs, double* us, double* X, double* U, void* stream)
{
    if (N < 0 || n_calls < 0 || n_modes < 0 || n_modes > kMaxModes) return 1;
    if (N == 0 || n_calls == 0) return 0;
    const int threads = 128;
    const int64_t blocks = (N + threads - 1) / threads;
    boris_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        N, n_calls, (float)L, (float)dt, qm, n_modes, ky, kz, psi, amp, xs, us, X, U);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
