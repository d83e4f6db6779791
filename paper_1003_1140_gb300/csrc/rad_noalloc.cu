// rad_noalloc.cu -- spectrum of one trajectory without any device allocation.
//
// For callers that are not allowed to allocate device memory themselves or
// through a library: for example a simulation code that hands all GPU memory
// to its own pool at start-up and forbids libraries from calling cudaMalloc,
// or a host application whose allocation calls are disabled.  The entry point
// runs the same ingest, FP32 split-phase accumulation and finalize as the
// context API, but takes all of its working memory from one fixed-size
// file-scope device array that every GPU loading this library holds until
// the process exits.  It calls no cudaMalloc, cudaFree or allocating library
// routine.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rad.h"
#include "rad_internal.cuh"

namespace {

using namespace rad;

// 96 MiB of working memory shared by every call on a device.
constexpr size_t kScratchBytes = size_t(96) << 20;
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// In host code the name g_scratch is only a host-side stand-in; kernels must
// be given the address cudaGetSymbolAddress returns on the device that is
// current.  It is looked up on every call (the lookup allocates nothing and
// costs microseconds): a cached address would go stale when the device's
// context is torn down and created again (cudaDeviceReset), and a kernel given
// it would fault.
cudaError_t scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

__global__ void noalloc_finalize(const double* acc, double* out, int64_t n, int coherent)
{
    const double pref = 1.0 / (4.0 * 3.14159265358979323846 * 3.14159265358979323846);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (coherent) {
            const double* a = acc + 4 * i;
            out[i] = pref * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
        } else {
            out[i] = pref * acc[i];
        }
    }
}

// Device (or managed) memory that kernels on device dev may dereference; host
// memory is refused before any launch instead of faulting inside one.
bool device_memory(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
    size_t off = 0;
    template <class T>
    size_t take(size_t count)
    {
        const size_t at = (off + 255) & ~size_t(255);
        off = at + count * sizeof(T);
        return at;
    }
};

}  // namespace

extern "C" int rad_spectrum_noalloc(const double* dirs, int32_t D, const double* freqs, int32_t F,
                                    double dt, double charge, int64_t N, int64_t n_calls,
                                    const double* x, const double* u, int32_t mode, double box_L,
                                    double* spectrum, void* cuda_stream)
{
    if (!dirs || D < 1 || !freqs || F < 1 || !(dt > 0.0) || !std::isfinite(dt) ||
        !std::isfinite(charge) || N < 1 || n_calls < 2 || !x || !u || !spectrum ||
        (mode != RAD_INCOHERENT && mode != RAD_COHERENT) || !(box_L >= 0.0) ||
        !std::isfinite(box_L))
        return RAD_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool coh = mode == RAD_COHERENT;

    // ---- layout (the same ring, anchor and accumulator formats as rad_init)
    constexpr int K = 32;
    const int64_t S = n_calls - 1;                       // samples: window [0, S)
    const int64_t ncols = (N + kTileP - 1) / kTileP * kTileP;
    const int64_t ring = (S + 31) / 32 * 32 + 64;
    const int64_t nblk = ring / K;
    const Accum32Config cfg{8, 0, K, coh, 2};
    const int ftl = 32 * cfg.ft;
    const int nft = (F + ftl - 1) / ftl;
    const int64_t ntiles = ncols / kTileP;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RAD_ECUDA;
    if (!device_memory(x, dev) || !device_memory(u, dev) || !device_memory(spectrum, dev))
        return RAD_EINVAL;
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (!accum32_dispatch(nullptr, cfg, 0, nullptr, &e, &nb) || nb < 1) return RAD_ECUDA;
    const int total_blocks = nb * sms;
    const double units = (double)ntiles * nft * D;
    const int G = (int)std::max(1.0, std::floor(units / (64.0 * total_blocks)));
    const int64_t ngroups = (ntiles + G - 1) / G;
    const int64_t n_items = ngroups * nft * D;
    if (n_items > INT32_MAX) return RAD_ENOSPACE;

    Carve cv;
    const size_t o_slab = cv.take<float>((size_t)ring * kCompsPlain * ncols);
    const size_t o_anc = cv.take<float>((size_t)nblk * 6 * ncols);
    const size_t o_state = cv.take<double>((size_t)9 * ncols);
    const size_t o_acc = cv.take<double>((size_t)D * F * (coh ? 4 : 1));
    const size_t o_dirs = cv.take<float>((size_t)D * 12);
    const size_t o_om = cv.take<float>((size_t)3 * F);
    const size_t o_win = cv.take<WinDev>(1);
    const size_t o_sp = cv.take<SpeciesDev>(1);
    const size_t o_items = cv.take<WorkItem>((size_t)n_items);
    const size_t o_ctr = cv.take<int>(2);
    if (cv.off > kScratchBytes) return RAD_ENOSPACE;

    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return RAD_ECUDA;
    unsigned char* B = static_cast<unsigned char*>(base);

    // ---- host tables, packed in the scratch's order and copied in one go
    const size_t t0 = o_dirs, t1 = o_ctr;
    std::vector<unsigned char> host(t1 - t0, 0);
    float* hd = reinterpret_cast<float*>(host.data() + (o_dirs - t0));
    for (int d = 0; d < D; ++d) {
        double n[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
        const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(l > 0.0) || !std::isfinite(l)) return RAD_EINVAL;
        for (int i = 0; i < 3; ++i) n[i] /= l;
        int k = 0;
        for (int i = 1; i < 3; ++i)
            if (std::fabs(n[i]) < std::fabs(n[k])) k = i;
        double ax[3] = {0, 0, 0};
        ax[k] = 1.0;
        double e1[3] = {n[1] * ax[2] - n[2] * ax[1], n[2] * ax[0] - n[0] * ax[2],
                        n[0] * ax[1] - n[1] * ax[0]};
        const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int i = 0; i < 3; ++i) e1[i] /= l1;
        const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2],
                              n[0] * e1[1] - n[1] * e1[0]};
        for (int i = 0; i < 3; ++i) {
            hd[12 * d + i] = (float)n[i];
            hd[12 * d + 3 + i] = (float)e1[i];
            hd[12 * d + 6 + i] = (float)e2[i];
            hd[12 * d + 9 + i] = (float)(n[i] - (double)(float)n[i]);
        }
    }
    float* ho = reinterpret_cast<float*>(host.data() + (o_om - t0));
    for (int k = 0; k < F; ++k) {
        if (!std::isfinite(freqs[k])) return RAD_EINVAL;
        const double nu = freqs[k] / 6.283185307179586476925286766559;
        ho[k] = (float)freqs[k];
        ho[F + k] = (float)nu;
        ho[2 * F + k] = (float)(nu - (double)(float)nu);
    }
    WinDev* hw = reinterpret_cast<WinDev*>(host.data() + (o_win - t0));
    hw->s0 = 0;
    hw->s1 = S;
    hw->grid_off = 0;
    hw->grid_len = F;
    hw->out_off = 0;
    hw->sel = -1;
    SpeciesDev* hs = reinterpret_cast<SpeciesDev*>(host.data() + (o_sp - t0));
    hs->qdt = charge * dt;
    hs->col0 = 0;
    hs->count = (int32_t)N;
    WorkItem* hi = reinterpret_cast<WorkItem*>(host.data() + (o_items - t0));
    int64_t ni = 0;
    for (int d = 0; d < D; ++d)
        for (int f = 0; f < nft; ++f)
            for (int64_t g = 0; g < ngroups; ++g)
                hi[ni++] = WorkItem{0, d, f, 0, (int32_t)(g * G),
                                    (int32_t)std::min<int64_t>(G, ntiles - g * G), d, 0};

#define NA_CU(call)                                   \
    do {                                              \
        if ((call) != cudaSuccess) return RAD_ECUDA;  \
    } while (0)
    NA_CU(cudaMemcpyAsync(B + t0, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    // what must start at zero: the accumulators, the item counter, the error word
    NA_CU(cudaMemsetAsync(B + o_acc, 0, (size_t)D * F * (coh ? 4 : 1) * sizeof(double), st));
    NA_CU(cudaMemsetAsync(B + o_ctr, 0, 2 * sizeof(int), st));
    int* counter = reinterpret_cast<int*>(B + o_ctr);
    int* err_word = counter + 1;

    IngestParams ip{};
    ip.x = x;
    ip.u = u;
    ip.n_in = N;
    ip.n_steps = (int32_t)n_calls;
    ip.step0 = 0;
    ip.dt = dt;
    ip.box_L = box_L;
    double* state = reinterpret_cast<double*>(B + o_state);
    ip.x_prev = state;
    ip.r_prev = state + 3 * ncols;
    ip.u_prev = state + 6 * ncols;
    ip.slab32 = reinterpret_cast<float*>(B + o_slab);
    ip.slab64 = nullptr;
    ip.anc32 = reinterpret_cast<float*>(B + o_anc);
    ip.ncols = ncols;
    ip.ring = ring;
    ip.comps = kCompsPlain;
    ip.K = K;
    ip.nblk = nblk;
    ip.n_species = 1;
    ip.in_off[0] = 0;
    ip.in_off[1] = N;
    ip.col_off[0] = 0;
    ip.check = 0;
    ip.err_word = err_word;
    NA_CU(launch_ingest(ip, st));

    Accum32Params ap{};
    ap.items = reinterpret_cast<const WorkItem*>(B + o_items);
    ap.n_items = (int32_t)n_items;
    ap.counter = counter;
    ap.wins = reinterpret_cast<const WinDev*>(B + o_win);
    ap.species = reinterpret_cast<const SpeciesDev*>(B + o_sp);
    ap.dirs32 = reinterpret_cast<const float*>(B + o_dirs);
    ap.omega = reinterpret_cast<const float*>(B + o_om);
    ap.nu_hi = ap.omega + F;
    ap.nu_lo = ap.omega + 2 * F;
    ap.slab32 = ip.slab32;
    ap.anc32 = ip.anc32;
    ap.ring = ring;
    ap.nblk = nblk;
    ap.comps = kCompsPlain;
    ap.dt_hi = (float)dt;
    ap.dt_lo = (float)(dt - (double)ap.dt_hi);
    ap.acc = reinterpret_cast<double*>(B + o_acc);
    ap.err_word = err_word;
    const int grid = (int)std::min<int64_t>(n_items, total_blocks);
    if (!accum32_dispatch(&ap, cfg, grid, st, &e, nullptr)) return RAD_ECUDA;
    NA_CU(e);

    const int64_t n_out = (int64_t)D * F;
    noalloc_finalize<<<(unsigned)std::min<int64_t>((n_out + 255) / 256, 4096), 256, 0, st>>>(
        ap.acc, spectrum, n_out, coh ? 1 : 0);
    NA_CU(cudaGetLastError());
    int errw = 0;
    NA_CU(cudaMemcpyAsync(&errw, err_word, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
#undef NA_CU
    return (errw & kErrTimeout) ? RAD_ETIMEOUT : RAD_OK;
}
