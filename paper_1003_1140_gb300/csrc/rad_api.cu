// rad_api.cu -- host side of the C ABI declared in include/rad.h.
//
// Owns the context: observer basis, frequency tables, species/column map,
// the trajectory ring and per-particle leapfrog state, the FP64 spectrum
// accumulators and the per-event work lists.  Every arithmetic step of the
// diagnostic runs in the kernels of rad_ingest.cu, rad_accum32.cuh (built in
// rad_accum32_ft*.cu), rad_accum64.cu and the finalize kernel below.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <sys/stat.h>
#include <map>
#include <string>
#include <vector>

#include "rad.h"
#include "rad_internal.cuh"

using namespace rad;

struct Event {
    int64_t call;                 // step after which the windows close
    std::vector<int> wins;
    std::vector<WorkItem> items;  // host copy
    WorkItem* d_items = nullptr;
};

// A replayable step: the ingest of one call, followed (for a closing step) by
// the accumulation of the windows that close there.
struct StepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ingest_node = nullptr;
};

// Failure-detection test hooks, read from the RAD_FAULT environment variable
// at rad_init (comma-separated tokens; unset or empty: none).  Every failure
// they cause is made on the host or by a bounded device wait:
//   alloc   rad_init fails as if the ring allocation had failed (RAD_ENOMEM)
//           after the tables are allocated, so the cleanup path runs;
//   graph   step-graph capture fails: the context falls back to direct
//           launches (rad_get_options then reports use_graph = 0);
//   step:N  the call starting at step N is lost once (it returns RAD_OK and
//           does nothing); the next call is refused with RAD_ESTEP and the
//           caller can hand step N over again;
//   stall   the next directly launched accumulation kernel holds block 0's
//           producer in a wait nothing ends, until the bounded wait expires:
//           the device error word is raised and rad_finalize returns
//           RAD_ETIMEOUT (once; rad_reset clears the error).
struct FaultHooks {
    bool alloc = false, graph = false, stall = false;
    int64_t drop_step = -1;
};

static bool parse_fault_env(FaultHooks& f)
{
    const char* env = std::getenv("RAD_FAULT");
    if (!env) return true;
    std::stringstream ss(env);
    std::string tok;
    while (std::getline(ss, tok, ',')) {
        if (tok.empty()) continue;
        if (tok == "alloc") {
            f.alloc = true;
        } else if (tok == "graph") {
            f.graph = true;
        } else if (tok == "stall") {
            f.stall = true;
        } else if (tok.compare(0, 5, "step:") == 0) {
            char* end = nullptr;
            const long long v = std::strtoll(tok.c_str() + 5, &end, 10);
            if (end == tok.c_str() + 5 || *end != '\0' || v < 0) return false;
            f.drop_step = v;
        } else {
            return false;
        }
    }
    return true;
}

// Internal status of graph_for: capture was not possible, launch directly.
constexpr int kGraphUnavailable = 1;

struct rad_ctx {
    // configuration
    int D = 0;
    int n_grids = 0;
    std::vector<int> grid_off, grid_len;
    std::vector<double> h_freqs;    // all frequency grids, concatenated
    double dt = 0.0, box_L = 0.0;
    int mode = 0, precision = 0;
    int n_species = 0;
    std::vector<rad_species> species;
    std::vector<int64_t> in_off;   // [n_species + 1]
    std::vector<int32_t> col_off;  // [n_species]
    int64_t n_in = 0, ncols = 0;
    std::vector<rad_window> wins;           // dir_set pointers are not kept (see win_dirs)
    std::vector<std::vector<int32_t>> win_dirs;   // per window: its directions, output order
    std::vector<int64_t> out_off;
    int64_t out_len = 0;
    rad_options opt{};
    Accum32Config cfg{8, 0, 16, false, 2};
    int K = 16;                    // anchor interval used by the ingest
    bool per_band_K = false;       // FP32 path: each frequency tile's anchor blocks are the
                                   // longest multiple K << m within the phase budget
    int nsub = 1;                  // sub-samples per PIC sample
    bool frozen = false;           // options frozen after the first step

    // device / stream
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;

    // ring
    int64_t ring = 0, nblk = 0;
    int comps = kCompsPlain;       // + the selector-flags word once selectors are defined;
                                   // kCompsPrec for the precise-phase variant
    float* slab32 = nullptr;
    double* slab64 = nullptr;
    float* anc32 = nullptr;
    double* x_prev = nullptr;
    double* r_prev = nullptr;
    double* u_prev = nullptr;

    // tables
    float* d_dirs32 = nullptr;
    double* d_dirs64 = nullptr;    // [D][9] n, e1, e2
    float* d_om32 = nullptr;
    float* d_nuhi = nullptr;
    float* d_nulo = nullptr;
    double* d_om64 = nullptr;
    WinDev* d_wins = nullptr;
    SelectorDev* d_sel = nullptr;
    int n_sel = 0;
    std::vector<int32_t> win_sel;
    SpeciesDev* d_species = nullptr;

    // accumulators
    double* acc = nullptr;       // [out_len] or [out_len][4]
    double* d_out = nullptr;     // scaled spectrum staging (device)
    int* d_err = nullptr;
    int* d_counter = nullptr;    // dynamic item counter of the FP32 kernel

    // staging for host inputs
    double* stage[2] = {nullptr, nullptr};
    int64_t stage_steps = 0;
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
    cudaEvent_t used_done[2] = {nullptr, nullptr};
    int stage_next = 0;
    // time-segmented ingest: per-segment image-count changes and staged state
    unsigned char* seg_buf = nullptr;
    size_t seg_bytes = 0;
    // blocked host path: per-block staging, per-(event, block) work lists
    double* bstage[2] = {nullptr, nullptr};
    size_t bstage_bytes = 0;
    int blk_count = 0;                               // blocks the lists were built for
    std::vector<std::vector<Event>> blk_events;      // [event][block]


    // events of the step axis
    std::vector<Event> events;     // eager: sorted by call; defer: one event
    std::map<int64_t, int> event_at;
    int64_t next_step = 0;
    int64_t max_s1 = 0;
    bool deferred_done = false;     // deferred windows already evaluated

    // timing
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> acc_ev, ing_ev;
    size_t acc_used = 0, ing_used = 0;
    int64_t acc_launches = 0, ing_launches = 0;
    bool time_ingest = false;

    // per-step CUDA graphs (use_graph option), by step kind: index 0 is a
    // plain step, 1 + e the step that closes event e
    std::vector<StepGraph> graphs;
    cudaStream_t cap_stream = nullptr;
    bool graph_off = false;        // capture failed once: direct launches only

    FaultHooks fault;

    std::string err;
};

static const char* kNoCtx = "null context";

static int fail(rad_ctx* c, int code, const char* fmt, ...)
{
    if (!c) return code;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, e_ == cudaErrorMemoryAllocation ? RAD_ENOMEM : RAD_ECUDA,    \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                \
    } while (0)

// ---------------------------------------------------------------------------
// finalize kernel: S = acc / (4 pi^2 c) (incoherent) or |sum A|^2 / (4 pi^2 c)
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const double* acc, double* out, int64_t n, int coherent)
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

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of the current device, or managed memory: what a kernel launched
// there may dereference.
static bool current_device_ptr(const void* p)
{
    int dev = -1;
    cudaPointerAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

static void basis(const double n[3], double e1[3], double e2[3])
{
    // e1 = normalise(n x a), a = the coordinate axis least aligned with n
    double ax[3] = {0, 0, 0};
    int k = 0;
    for (int i = 1; i < 3; ++i)
        if (std::fabs(n[i]) < std::fabs(n[k])) k = i;
    ax[k] = 1.0;
    double c[3] = {n[1] * ax[2] - n[2] * ax[1], n[2] * ax[0] - n[0] * ax[2],
                   n[0] * ax[1] - n[1] * ax[0]};
    double l = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    for (int i = 0; i < 3; ++i) e1[i] = c[i] / l;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
}

bool rad::accum32_dispatch(const Accum32Params* p, const Accum32Config& cfg, int grid,
                           cudaStream_t st, cudaError_t* err, int* nb)
{
    if (cfg.pm) return accum32_precise(p, cfg, grid, st, err, nb);
    if (cfg.band) return accum32_band(p, cfg, grid, st, err, nb);
    return accum32_ft8_sfu(p, cfg, grid, st, err, nb) || accum32_ft8_mix(p, cfg, grid, st, err, nb) ||
           accum32_ft16(p, cfg, grid, st, err, nb) || accum32_ft4(p, cfg, grid, st, err, nb);
}

static int chunk_len(const rad_ctx* c) { return c->precision == RAD_FP64 ? kChunk64 : kChunk32; }

static int freq_tile(const rad_ctx* c)
{
    return c->precision == RAD_FP64 ? 32 * accum64_ft() : 32 * c->cfg.ft;
}

static std::vector<std::vector<int>> band_kmul(const rad_ctx* c, int ftl);
static std::vector<std::vector<int>> precise_tiles(const rad_ctx* c);

// Build the work items of one event (set of windows) and sort them by cost;
// with `ranges` only the particle tiles [first, second) of each species (the
// blocked host path), the groups sized for those tiles so that every list
// balances over the GPU.
static void build_items(rad_ctx* c, Event& ev, int total_blocks,
                        const std::vector<std::pair<int, int>>* ranges = nullptr)
{
    auto lo_of = [&](int s) { return ranges ? (*ranges)[s].first : 0; };
    auto hi_of = [&](int s) { return ranges ? (*ranges)[s].second : INT_MAX; };
    const int ftl = freq_tile(c);
    const int ch = chunk_len(c);
    // total (tile x direction x ftile) units, to size the particle groups
    double units = 0;
    for (int w : ev.wins) {
        const rad_window& W = c->wins[w];
        const int nft = (c->grid_len[W.freq_grid] + ftl - 1) / ftl;
        for (int s = 0; s < c->n_species; ++s)
            if ((W.species_mask >> s) & 1u) {
                const int nts = (int)((c->species[s].count + kTileP - 1) / kTileP);
                const int in_range = std::max(0, std::min(nts, hi_of(s)) - std::max(0, lo_of(s)));
                units += (double)in_range * nft * c->win_dirs[w].size();
            }
    }
    // about 256 items per resident block: the launch ends with every block on its
    // last item, so an item's length is the tail's scale (1/256 of a block's
    // work); an item costs one list fetch and one FP64 flush of its sums
    const double target_items = 256.0 * std::max(1, total_blocks);
    int G = (int)std::max(1.0, std::floor(units / target_items));
    const std::vector<std::vector<int>> km = band_kmul(c, ftl);
    const std::vector<std::vector<int>> pt = precise_tiles(c);
    ev.items.clear();
    std::vector<int64_t> cost;
    for (int w : ev.wins) {
        const rad_window& W = c->wins[w];
        if (W.s1 <= W.s0) continue;
        const int nft = (c->grid_len[W.freq_grid] + ftl - 1) / ftl;
        const int64_t nch = (W.s1 * c->nsub - 1) / ch - W.s0 * c->nsub / ch + 1;
        for (int s = 0; s < c->n_species; ++s) {
            if (!((W.species_mask >> s) & 1u) || c->species[s].count == 0) continue;
            const int nt = (int)((c->species[s].count + kTileP - 1) / kTileP);
            const int t_end = std::min(nt, hi_of(s));
            // tile-group-major: the items that read the same particles
            // (all directions and frequency tiles) are adjacent in the list,
            // so they run at about the same time and share L2
            const std::vector<int32_t>& wd = c->win_dirs[w];
            for (int t0 = std::max(0, lo_of(s)); t0 < t_end; t0 += G)
                for (int row = 0; row < (int)wd.size(); ++row)
                    for (int f = 0; f < nft; ++f) {
                        WorkItem it{w, wd[row], f, s, t0, std::min(G, t_end - t0), row,
                                    km[W.freq_grid][f],
                                    c->cfg.pm == 2 ? pt[W.freq_grid][f] : 0};
                        ev.items.push_back(it);
                        cost.push_back((int64_t)it.ntiles * nch);
                    }
        }
    }
    std::vector<size_t> ord(ev.items.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<WorkItem> sorted(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = ev.items[ord[i]];
    ev.items.swap(sorted);
}

static int blocks_per_sm(const rad_ctx* c)
{
    if (c->precision == RAD_FP64) return std::max(1, accum64_blocks_per_sm(c->mode == RAD_COHERENT));
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (!accum32_dispatch(nullptr, c->cfg, 0, nullptr, &e, &nb)) return 0;
    return nb;
}

static cudaEvent_t next_event(std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& pool, size_t& used,
                              bool start)
{
    if (start) {
        if (used == pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            pool.push_back({a, b});
        }
        return pool[used].first;
    }
    return pool[used++].second;
}

// ---------------------------------------------------------------------------
// autotuner for the FP32 kernel variant (variant = RAD_VARIANT_AUTO)
// ---------------------------------------------------------------------------
// Largest anchor interval K whose worst-case rounding of the offset phase per
// update, w_max * |dphi|_max * 2^-24, stays within the phase budget (1e-4 rad
// unless the options give one); the offsets are centred in their block, so
// |dphi| <= (K - 1) dt (1 - n.beta) / 2 <= (K - 1) dt.  (The special-function
// unit's own reduction of the radian argument adds about 1.3e-7 |theta| rad,
// and the FP32 roundings of w and dphi add errors of the same order, all
// proportional to |dphi|.)
static double phase_budget(const rad_ctx* c)
{
    return c->opt.reserved[3] > 0 ? c->opt.reserved[3] * 1e-9 : 1e-4;
}

static int budget_K_at(const rad_ctx* c, double wmax)
{
    for (int K : {32, 16}) {
        const double err = wmax * (K - 1) * (c->dt / c->nsub) * std::ldexp(1.0, -24);
        if (err <= phase_budget(c)) return K;
    }
    return 8;
}

static int budget_K(const rad_ctx* c)
{
    double wmax = 0.0;
    for (int g = 0; g < c->n_grids; ++g)
        for (int k = 0; k < c->grid_len[g]; ++k)
            wmax = std::max(wmax, std::fabs(c->h_freqs[c->grid_off[g] + k]));
    return budget_K_at(c, wmax);
}

// Per frequency tile of each grid, the anchor blocks' multiple of the ring's K
// (as a shift): the longest interval K << m, up to one chunk, within the phase
// budget at the tile's highest frequency.  The ring is anchored at the K of the
// highest frequency of all grids, so a lower band takes fewer, longer blocks.
// All zero unless the context chose its K by the budget.
static std::vector<std::vector<int>> band_kmul(const rad_ctx* c, int ftl)
{
    std::vector<std::vector<int>> km(c->n_grids);
    for (int g = 0; g < c->n_grids; ++g) {
        const int nft = (c->grid_len[g] + ftl - 1) / ftl;
        km[g].assign(nft, 0);
        if (!c->per_band_K) continue;
        for (int f = 0; f < nft; ++f) {
            double wmax = 0.0;
            for (int k = f * ftl; k < std::min((f + 1) * ftl, c->grid_len[g]); ++k)
                wmax = std::max(wmax, std::fabs(c->h_freqs[c->grid_off[g] + k]));
            const int Kt = std::min(budget_K_at(c, wmax), kChunk32);
            while ((c->K << (km[g][f] + 1)) <= Kt) ++km[g][f];
        }
    }
    return km;
}

static std::string tune_cache_path()
{
    if (const char* e = std::getenv("RAD_AUTOTUNE_CACHE")) return e;
    if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/rad_gb300_autotune.tsv";
    return "";
}

static std::string tune_key(const rad_ctx* c, int K)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    std::ostringstream k;
    k << prop.name << "|sm" << c->sms << "|D" << c->D << "|m" << c->mode << "|K" << K << "|g";
    for (int g = 0; g < c->n_grids; ++g) k << c->grid_len[g] << ",";
    k << "|s";
    for (const auto& sp : c->species) k << sp.count << ",";
    k << "|w";
    for (size_t w = 0; w < c->wins.size(); ++w) {
        const auto& W = c->wins[w];
        k << (W.s1 - W.s0) << ":" << W.species_mask << ":" << W.freq_grid << ":"
          << c->win_dirs[w].size() << ",";
    }
    k << "|d" << c->opt.defer << "|n" << std::max(1, c->opt.subcycle) << "|b" << c->cfg.band
      << "|p" << c->cfg.pm;
    return k.str();
}

static bool tune_lookup(const std::string& key, Accum32Config& cfg)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        const size_t tab = line.find('\t');
        if (tab == std::string::npos || line.compare(0, tab, key) != 0 || tab != key.size()) continue;
        std::istringstream v(line.substr(tab + 1));
        int ft, np, K, mb;
        if (v >> ft >> np >> K >> mb) {
            cfg.ft = ft;
            cfg.np = np;
            cfg.K = K;
            cfg.mb = mb;
            found = true;   // the last entry for a key wins
        }
    }
    return found;
}

static void tune_store(const std::string& key, const Accum32Config& cfg)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
    std::ofstream f(path, std::ios::app);
    if (f) f << key << '\t' << cfg.ft << ' ' << cfg.np << ' ' << cfg.K << ' ' << cfg.mb << '\n';
}

static int blocks_per_sm(const rad_ctx* c);

// The autotuner's timing slice: n single-tile items (one particle tile, one
// direction, one frequency tile, the whole window) of the window with the most
// samples x frequencies, so that every candidate times the same kind of work
// and the slice stays a few tens of milliseconds whatever the workload's size.
static void tune_slice(const rad_ctx* c, Event& ev, size_t n)
{
    ev.items.clear();
    int best = -1;
    double cost = 0.0;
    for (size_t w = 0; w < c->wins.size(); ++w) {
        const rad_window& W = c->wins[w];
        int64_t np = 0;
        for (int s = 0; s < c->n_species; ++s)
            if ((W.species_mask >> s) & 1u) np += c->species[s].count;
        const double cw = (double)(W.s1 - W.s0) * c->grid_len[W.freq_grid];
        if (W.s1 > W.s0 && np > 0 && cw > cost) {
            cost = cw;
            best = (int)w;
        }
    }
    if (best < 0) return;
    const rad_window& W = c->wins[best];
    const int ftl = freq_tile(c);
    const int nft = (c->grid_len[W.freq_grid] + ftl - 1) / ftl;
    const std::vector<std::vector<int>> km = band_kmul(c, ftl);
    const std::vector<std::vector<int>> pt = precise_tiles(c);
    const std::vector<int32_t>& wd = c->win_dirs[best];
    for (int s = 0; s < c->n_species && ev.items.size() < n; ++s) {
        if (!((W.species_mask >> s) & 1u)) continue;
        const int nt = (int)((c->species[s].count + kTileP - 1) / kTileP);
        for (int t = 0; t < nt && ev.items.size() < n; ++t)
            for (int row = 0; row < (int)wd.size() && ev.items.size() < n; ++row)
                for (int f = 0; f < nft && ev.items.size() < n; ++f)
                    ev.items.push_back(WorkItem{best, wd[row], f, s, t, 1, row, km[W.freq_grid][f],
                                                c->cfg.pm == 2 ? pt[W.freq_grid][f] : 0});
    }
}

// Time the candidate variants on a slice of single-tile items (the ring's
// contents do not change the kernel's instruction stream) and keep the fastest.
static int autotune32(rad_ctx* c, int K)
{
    const std::string key = tune_key(c, K);
    Accum32Config best = c->cfg;
    best.K = K;
    if (tune_lookup(key, best)) {
        c->cfg = best;
        c->cfg.coh = c->mode == RAD_COHERENT;
        return RAD_OK;
    }
    const bool coh = c->mode == RAD_COHERENT;
    std::vector<Accum32Config> cands = {{8, 0, K, coh, 2}, {8, 0, K, coh, 3}, {8, 1, K, coh, 2},
                                        {8, 1, K, coh, 3}, {8, 2, K, coh, 2}, {4, 0, K, coh, 4}};
    if (c->cfg.band) cands = {{8, 0, K, coh, 2, true}, {8, 0, K, coh, 3, true}};
    if (c->cfg.pm) cands = {{8, 0, K, coh, 2, false, c->cfg.pm}, {8, 0, K, coh, 3, false, c->cfg.pm}};
    // small problems: not worth timing
    if (rad_updates(c) < (int64_t)2e10) {
        c->cfg = cands[0];
        return RAD_OK;
    }
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (const auto& cand : cands) {
        c->cfg = cand;
        const int bps = blocks_per_sm(c);
        if (bps < 1) continue;
        const int total_blocks = bps * c->sms;
        Event ev;
        tune_slice(c, ev, (size_t)16 * total_blocks);
        const size_t n = ev.items.size();
        if (n == 0) continue;
        WorkItem* d_items = nullptr;
        CU(cudaMalloc(&d_items, n * sizeof(WorkItem)));
        CU(cudaMemcpy(d_items, ev.items.data(), n * sizeof(WorkItem), cudaMemcpyHostToDevice));
        Accum32Params p{};
        p.items = d_items;
        p.n_items = (int32_t)n;
        p.counter = c->d_counter;
        p.wins = c->d_wins;
        p.species = c->d_species;
        p.dirs32 = c->d_dirs32;
        p.omega = c->d_om32;
        p.nu_hi = c->d_nuhi;
        p.nu_lo = c->d_nulo;
        p.slab32 = c->slab32;
        p.anc32 = c->anc32;
        p.ring = c->ring;
        p.nblk = c->nblk;
        p.comps = c->comps;
        p.dt_hi = (float)(c->dt / c->nsub);
        p.dt_lo = (float)(c->dt / c->nsub - (double)p.dt_hi);
        p.acc = c->acc;
        p.err_word = c->d_err;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CU(cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->stream));
            CU(cudaEventRecord(e0, c->stream));
            cudaError_t e = cudaSuccess;
            accum32_dispatch(&p, cand, (int)std::min<size_t>(n, total_blocks), c->stream, &e, nullptr);
            CU(e);
            CU(cudaEventRecord(e1, c->stream));
            CU(cudaEventSynchronize(e1));
            float ms = 0;
            CU(cudaEventElapsedTime(&ms, e0, e1));
            // per particle tile x frequency (an item covers 32 ft frequencies of one
            // tile), so candidates with different item sizes and numbers of
            // resident blocks compare fairly
            ms_min = std::min(ms_min, ms / ((float)n * (float)cand.ft));
        }
        cudaFree(d_items);
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timing launches may have added (zero or stale) terms: start clean
    const size_t acc_n = (size_t)c->out_len * (coh ? 4 : 1);
    CU(cudaMemsetAsync(c->acc, 0, std::max<size_t>(1, acc_n) * sizeof(double), c->stream));
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->cfg = best;
    tune_store(key, best);
    return RAD_OK;
}

// Per frequency tile (8 frequencies per thread) of each grid, whether the
// precise-phase variant takes it: every tile, or with a phase budget the tiles
// whose rounding bound at K = 32, w_max 31 dt 2^-24, exceeds the budget.
static std::vector<std::vector<int>> precise_tiles(const rad_ctx* c)
{
    std::vector<std::vector<int>> pt(c->n_grids);
    const int ftl = 32 * 8;
    const double dts = c->dt / std::max(1, c->opt.subcycle);
    for (int g = 0; g < c->n_grids; ++g) {
        const int nft = (c->grid_len[g] + ftl - 1) / ftl;
        pt[g].assign(nft, 1);
        if (c->opt.reserved[3] <= 0) continue;
        for (int f = 0; f < nft; ++f) {
            double wmax = 0.0;
            for (int k = f * ftl; k < std::min((f + 1) * ftl, c->grid_len[g]); ++k)
                wmax = std::max(wmax, std::fabs(c->h_freqs[c->grid_off[g] + k]));
            pt[g][f] = wmax * 31.0 * dts * std::ldexp(1.0, -24) > phase_budget(c);
        }
    }
    return pt;
}

// The precise-phase build: 0 none, 1 every item, 2 the items of precise tiles.
static int precise_mode(const rad_ctx* c)
{
    if (c->precision != RAD_FP32_SPLIT || c->opt.variant != RAD_VARIANT_PRECISE) return 0;
    bool any = false, all = true;
    for (const auto& g : precise_tiles(c))
        for (int v : g) {
            any = any || v;
            all = all && v;
        }
    return all ? 1 : (any ? 2 : 0);
}

// Freeze options: pick K / FT, build events and their item lists.
static int freeze(rad_ctx* c)
{
    if (c->frozen) return RAD_OK;
    CU(cudaSetDevice(c->device));
    const int pm = precise_mode(c);
    if (pm && c->comps != kCompsPrec) {
        // the precise-phase ring also carries the lo part of each position offset
        CU(cudaFree(c->slab32));
        c->slab32 = nullptr;
        c->comps = kCompsPrec;
        const size_t bytes = (size_t)c->ring * c->comps * c->ncols * sizeof(float);
        CU(cudaMalloc(&c->slab32, bytes));
        CU(cudaMemset(c->slab32, 0, bytes));
    }
    if (c->opt.subcycle > 1 && c->nsub == 1) {
        // sub-cycling: the ring holds nsub samples per PIC sample, windows and
        // the per-sample weight dt are in sub-sample units
        c->nsub = c->opt.subcycle;
        const int64_t nc = c->ncols;
        const size_t es = c->precision == RAD_FP64 ? sizeof(double) : sizeof(float);
        void*& slab = c->precision == RAD_FP64 ? reinterpret_cast<void*&>(c->slab64)
                                               : reinterpret_cast<void*&>(c->slab32);
        CU(cudaFree(slab));
        slab = nullptr;
        c->ring *= c->nsub;
        CU(cudaMalloc(&slab, (size_t)c->ring * c->comps * nc * es));
        CU(cudaMemset(slab, 0, (size_t)c->ring * c->comps * nc * es));
        std::vector<WinDev> wd(c->wins.size());
        CU(cudaMemcpy(wd.data(), c->d_wins, wd.size() * sizeof(WinDev), cudaMemcpyDeviceToHost));
        for (size_t w = 0; w < wd.size(); ++w) {
            wd[w].s0 = c->wins[w].s0 * c->nsub;
            wd[w].s1 = c->wins[w].s1 * c->nsub;
        }
        CU(cudaMemcpy(c->d_wins, wd.data(), wd.size() * sizeof(WinDev), cudaMemcpyHostToDevice));
        std::vector<SpeciesDev> sd(c->n_species);
        CU(cudaMemcpy(sd.data(), c->d_species, sd.size() * sizeof(SpeciesDev), cudaMemcpyDeviceToHost));
        for (int s = 0; s < c->n_species; ++s) sd[s].qdt = c->species[s].charge * c->dt / c->nsub;
        CU(cudaMemcpy(c->d_species, sd.data(), sd.size() * sizeof(SpeciesDev), cudaMemcpyHostToDevice));
    }
    if (c->precision == RAD_FP32_SPLIT) {
        c->K = c->opt.anchor_K ? c->opt.anchor_K : 32;
        c->cfg.K = c->K;
        c->cfg.ft = c->opt.freq_per_lane ? c->opt.freq_per_lane : 8;
        c->cfg.np = c->opt.variant == RAD_VARIANT_MIX ? (c->cfg.ft == 8 ? 2 : 4) : 0;
        if (c->opt.variant == RAD_VARIANT_MIX && c->opt.reserved[1] > 0) c->cfg.np = c->opt.reserved[1];
        c->cfg.coh = c->mode == RAD_COHERENT;
        c->cfg.mb = c->opt.blocks_per_sm ? c->opt.blocks_per_sm : 2;
        if (c->cfg.ft == 16 && c->cfg.mb != 2)
            return fail(c, RAD_EINVAL, "16 frequencies per thread is built for 2 blocks per SM only");
        if (c->cfg.ft == 4 && (c->cfg.mb != 4 || c->cfg.np != 0))
            return fail(c, RAD_EINVAL, "4 frequencies per thread is built for 4 blocks per SM, SFU only");
        if (c->cfg.ft == 8 && c->cfg.mb == 4)
            return fail(c, RAD_EINVAL, "8 frequencies per thread is built for 2 or 3 blocks per SM");
        const bool prec = pm != 0;
        c->cfg.pm = pm;
        if (prec) {
            // one turn of phase per update regardless of K: the ring's anchor
            // interval stays at 32
            c->K = 32;
            c->cfg.K = 32;
        }
        const bool tune = (c->opt.variant == RAD_VARIANT_AUTO ||
                           c->opt.variant == RAD_VARIANT_PRECISE) &&
                          !c->opt.freq_per_lane && !c->opt.blocks_per_sm;
        c->per_band_K = false;
        if (!prec && !c->opt.anchor_K && (tune || c->opt.reserved[3] > 0)) {
            c->K = budget_K(c);
            c->cfg.K = c->K;
            // longer anchor blocks for the lower bands where any frequency tile
            // can take one: the 8-SFU-frequency build with per-item blocks
            if (tune || (c->cfg.ft == 8 && c->cfg.np == 0)) {
                c->per_band_K = true;
                bool any = false;
                for (const auto& g : band_kmul(c, 32 * 8))
                    for (int m : g) any = any || m > 0;
                c->per_band_K = any;
            }
        }
        c->cfg.band = c->per_band_K;
        if (c->per_band_K) {
            c->cfg.ft = 8;
            c->cfg.np = 0;
        }
        // anchor positions: one FP32 hi/lo 3-vector per particle per K samples of the ring
        c->nblk = c->ring / c->K;
        if (!c->anc32) {
            CU(cudaMalloc(&c->anc32, (size_t)c->nblk * 6 * c->ncols * sizeof(float)));
            CU(cudaMemset(c->anc32, 0, (size_t)c->nblk * 6 * c->ncols * sizeof(float)));
        }
        if (tune) {
            const int rc = autotune32(c, c->K);
            if (rc) return rc;
        }
    }
    // events
    c->events.clear();
    c->event_at.clear();
    if (c->opt.defer) {
        Event ev;
        ev.call = -1;
        for (size_t w = 0; w < c->wins.size(); ++w) ev.wins.push_back((int)w);
        c->events.push_back(ev);
    } else {
        std::map<int64_t, std::vector<int>> by;
        for (size_t w = 0; w < c->wins.size(); ++w)
            if (c->wins[w].s1 > c->wins[w].s0) by[c->wins[w].s1].push_back((int)w);
        for (auto& kv : by) {
            Event ev;
            ev.call = kv.first;
            ev.wins = kv.second;
            c->event_at[kv.first] = (int)c->events.size();
            c->events.push_back(ev);
        }
    }
    const int bps = blocks_per_sm(c);
    if (bps < 1) return fail(c, RAD_EINVAL, "the selected kernel variant cannot be resident");
    const int total_blocks = bps * c->sms;
    for (auto& ev : c->events) {
        build_items(c, ev, total_blocks);
        if (!ev.items.empty()) {
            CU(cudaMalloc(&ev.d_items, ev.items.size() * sizeof(WorkItem)));
            CU(cudaMemcpy(ev.d_items, ev.items.data(), ev.items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice));
        }
    }
    c->frozen = true;
    return RAD_OK;
}

// The stall hook applies to one launch only.
static int32_t take_stall(rad_ctx* c)
{
    const bool s = c->fault.stall;
    c->fault.stall = false;
    return s ? 1 : 0;
}

static int launch_event(rad_ctx* c, Event& ev)
{
    if (ev.items.empty()) return RAD_OK;
    const int total_blocks = blocks_per_sm(c) * c->sms;
    const int grid = (int)std::min<int64_t>((int64_t)ev.items.size(), total_blocks);
    cudaEvent_t e0 = next_event(c->acc_ev, c->acc_used, true);
    CU(cudaEventRecord(e0, c->stream));
    cudaError_t e;
    if (c->precision == RAD_FP64) {
        Accum64Params p{};
        p.items = ev.d_items;
        p.n_items = (int32_t)ev.items.size();
        p.wins = c->d_wins;
        p.species = c->d_species;
        p.dirs64 = c->d_dirs64;
        p.omega = c->d_om64;
        p.slab64 = c->slab64;
        p.ring = c->ring;
        p.comps = c->comps;
        p.dt = c->dt / c->nsub;
        p.acc = c->acc;
        p.err_word = c->d_err;
        p.fault_stall = take_stall(c);
        e = launch_accum64(p, c->mode == RAD_COHERENT, grid, c->stream);
    } else {
        Accum32Params p{};
        p.items = ev.d_items;
        p.n_items = (int32_t)ev.items.size();
        p.counter = c->d_counter;
        p.wins = c->d_wins;
        p.species = c->d_species;
        p.dirs32 = c->d_dirs32;
        p.omega = c->d_om32;
        p.nu_hi = c->d_nuhi;
        p.nu_lo = c->d_nulo;
        p.slab32 = c->slab32;
        p.anc32 = c->anc32;
        p.ring = c->ring;
        p.nblk = c->nblk;
        p.comps = c->comps;
        p.dt_hi = (float)(c->dt / c->nsub);
        p.dt_lo = (float)(c->dt / c->nsub - (double)p.dt_hi);
        p.acc = c->acc;
        p.err_word = c->d_err;
        p.fault_stall = take_stall(c);
        CU(cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->stream));
        e = cudaSuccess;
        if (!accum32_dispatch(&p, c->cfg, grid, c->stream, &e, nullptr))
            return fail(c, RAD_EINVAL, "kernel variant not built");
    }
    if (e != cudaSuccess) return fail(c, RAD_ECUDA, "accumulation launch failed: %s", cudaGetErrorString(e));
    cudaEvent_t e1 = next_event(c->acc_ev, c->acc_used, false);
    CU(cudaEventRecord(e1, c->stream));
    ++c->acc_launches;
    return RAD_OK;
}

// The context's part of an ingest launch (inputs, step range and particle
// range are the caller's).
static IngestParams ingest_params(const rad_ctx* c)
{
    IngestParams p{};
    p.n_in = c->n_in;
    p.dt = c->dt;
    p.box_L = c->box_L;
    p.x_prev = c->x_prev;
    p.r_prev = c->r_prev;
    p.u_prev = c->u_prev;
    p.slab32 = c->slab32;
    p.slab64 = c->slab64;
    p.anc32 = c->anc32;
    p.ncols = c->ncols;
    p.ring = c->ring;
    p.comps = c->comps;
    p.K = c->K;
    p.nblk = c->nblk;
    p.n_species = c->n_species;
    for (int s = 0; s <= c->n_species; ++s) p.in_off[s] = c->in_off[s];
    for (int s = 0; s < c->n_species; ++s) p.col_off[s] = c->col_off[s];
    p.check = c->opt.check_inputs;
    p.err_word = c->d_err;
    p.sel = c->d_sel;
    p.n_sel = c->n_sel;
    p.nsub = c->nsub;
    return p;
}

// Scratch of a time-segmented ingest launch over count particles and n_steps
// calls (segments of kSegLen calls, a multiple of every anchor interval).
constexpr int kSegLen = 64;
static int seg_scratch(rad_ctx* c, int64_t count, int64_t n_steps, IngestParams& p)
{
    const int64_t nseg_max = std::min<int64_t>(n_steps / kSegLen + 2, 257);   // launch_ingest caps at 256
    const size_t sb = (size_t)9 * count * sizeof(double);
    const size_t wb = (size_t)nseg_max * 3 * count * sizeof(int32_t);
    if (c->seg_bytes < sb + wb) {
        if (c->seg_buf) {
            CU(cudaStreamSynchronize(c->stream));
            CU(cudaFree(c->seg_buf));
            c->seg_buf = nullptr;
            c->seg_bytes = 0;
        }
        CU(cudaMalloc(&c->seg_buf, sb + wb));
        c->seg_bytes = sb + wb;
    }
    p.state_out = reinterpret_cast<double*>(c->seg_buf);
    p.wind = reinterpret_cast<int32_t*>(c->seg_buf + sb);
    p.seg_len = kSegLen;
    return RAD_OK;
}

// Ingest n steps from device arrays x, u ([n][3][n_in]) starting at step0.
static int ingest_device(rad_ctx* c, int64_t step0, int64_t n, const double* x, const double* u)
{
    IngestParams p = ingest_params(c);
    int64_t s = step0;
    const int64_t end = step0 + n;
    while (s < end) {
        // split at the next closing call so windows close right after their last sample
        int64_t stop = end;
        if (!c->opt.defer) {
            auto itv = c->event_at.lower_bound(s);
            if (itv != c->event_at.end() && itv->first < end) stop = itv->first + 1;
        }
        p.x = x + (s - step0) * 3 * c->n_in;
        p.u = u + (s - step0) * 3 * c->n_in;
        p.step0 = s;
        p.n_steps = (int32_t)(stop - s);
        int rs = seg_scratch(c, c->n_in, stop - s, p);
        if (rs) return rs;
        cudaEvent_t e0 = nullptr;
        if (c->time_ingest) {
            e0 = next_event(c->ing_ev, c->ing_used, true);
            CU(cudaEventRecord(e0, c->stream));
        }
        cudaError_t e = launch_ingest(p, c->stream);
        if (e != cudaSuccess) return fail(c, RAD_ECUDA, "ingest launch failed: %s", cudaGetErrorString(e));
        if (c->time_ingest) CU(cudaEventRecord(next_event(c->ing_ev, c->ing_used, false), c->stream));
        ++c->ing_launches;
        if (!c->opt.defer) {
            auto itv = c->event_at.find(stop - 1);
            if (itv != c->event_at.end()) {
                int rc = launch_event(c, c->events[itv->second]);
                if (rc) return rc;
            }
        }
        s = stop;
    }
    return RAD_OK;
}

// Host inputs, eager windows: the particle axis is cut into a few
// blocks of whole tiles.  Each block's share of the call's steps is copied
// (pitched copies on the copy stream, double-buffered) and ingested on its own,
// and at every window close only that block's work items are launched.  The
// copies of block b + 1 run while block b is ingested and accumulated, so the
// transfer hides behind the accumulation instead of preceding it.  Per-particle
// ingest state makes the blocks independent; each block's ring columns are
// read by its own accumulation before its next segment is ingested.  Blocks
// grow geometrically (1/32 of the tiles, then x4): only the first, small
// block's transfer is exposed, and each later transfer (4x the previous block's
// particles, at ~1/8 of its accumulation time per particle) fits behind it.
constexpr int kHostBlocks = 4;      // gates the path: n_in >= 64 tiles per block
// per staging buffer: a whole block of a long call fits (the largest block of
// 65,536 particles x 4097 calls: 6.4 GB), so block b + 1 is copied entirely while block b is
// accumulated; longer segments arrive in chunks, whose last copy waits for the
// block's first ingest
constexpr size_t kBlockStageBytes = size_t(8) << 30;

// Tile boundaries of the blocks: 1/32 of the tiles, then each block 4x the
// previous one, the remainder merged into the last block when it is small.
static std::vector<int> block_bounds(int nt)
{
    std::vector<int> b = {0};
    int cur = std::max(1, nt / 32);
    while (b.back() < nt) {
        int next = std::min(nt, b.back() + cur);
        if (nt - next < cur / 2) next = nt;
        b.push_back(next);
        cur *= 4;
    }
    return b;
}

// Tile boundaries of the blocks for every species: the geometric schedule of
// the whole particle axis applied to each species in proportion.
static std::vector<std::vector<int>> species_bounds(const rad_ctx* c)
{
    int nt_all = 0;
    std::vector<int> nts(c->n_species);
    for (int s = 0; s < c->n_species; ++s) {
        nts[s] = (int)((c->species[s].count + kTileP - 1) / kTileP);
        nt_all += nts[s];
    }
    const std::vector<int> g = block_bounds(std::max(1, nt_all));
    std::vector<std::vector<int>> b(c->n_species);
    for (int s = 0; s < c->n_species; ++s) {
        b[s].resize(g.size());
        for (size_t i = 0; i < g.size(); ++i)
            b[s][i] = i + 1 == g.size() ? nts[s] : (int)((int64_t)g[i] * nts[s] / nt_all);
    }
    return b;
}

static int blocked_lists(rad_ctx* c, const std::vector<std::vector<int>>& bounds)
{
    const int nblocks = (int)bounds[0].size() - 1;
    if (c->blk_count == nblocks) return RAD_OK;
    for (auto& row : c->blk_events)
        for (auto& ev : row) cudaFree(ev.d_items);
    c->blk_events.assign(c->events.size(), std::vector<Event>(nblocks));
    const int total_blocks = blocks_per_sm(c) * c->sms;
    for (size_t e = 0; e < c->events.size(); ++e)
        for (int b = 0; b < nblocks; ++b) {
            Event& ev = c->blk_events[e][b];
            ev.call = c->events[e].call;
            ev.wins = c->events[e].wins;
            std::vector<std::pair<int, int>> ranges(c->n_species);
            for (int s = 0; s < c->n_species; ++s) ranges[s] = {bounds[s][b], bounds[s][b + 1]};
            build_items(c, ev, total_blocks, &ranges);
            if (!ev.items.empty()) {
                CU(cudaMalloc(&ev.d_items, ev.items.size() * sizeof(WorkItem)));
                CU(cudaMemcpy(ev.d_items, ev.items.data(), ev.items.size() * sizeof(WorkItem),
                              cudaMemcpyHostToDevice));
            }
        }
    c->blk_count = nblocks;
    return RAD_OK;
}

// The blocked path (see above).  Ingest and accumulation stay in order on the
// context's stream; only the copies run ahead on the copy stream.  (Ingesting
// block b + 1 on a second stream during block b's accumulation, or blocking
// device-resident inputs too, measured slower: the extra launch tails cost more
// than the overlap saves.)
static int ingest_host_blocked(rad_ctx* c, int64_t step0, int64_t n, const double* x,
                               const double* u)
{
    const int64_t N = c->n_in;
    const int S = c->n_species;
    const std::vector<std::vector<int>> bounds = species_bounds(c);
    const int nblocks = (int)bounds[0].size() - 1;
    // particles of species s in block b: species-local [lo, hi)
    auto range = [&](int s, int b, int64_t& lo, int64_t& cnt) {
        lo = (int64_t)bounds[s][b] * kTileP;
        cnt = std::max<int64_t>(0, std::min<int64_t>((int64_t)bounds[s][b + 1] * kTileP,
                                                     c->species[s].count) - lo);
    };
    int64_t ppb = 1;                                                  // largest block
    for (int b = 0; b < nblocks; ++b) {
        int64_t tot = 0;
        for (int s = 0; s < S; ++s) {
            int64_t lo, cnt;
            range(s, b, lo, cnt);
            tot += cnt;
        }
        ppb = std::max(ppb, tot);
    }
    int rc = blocked_lists(c, bounds);
    if (rc) return rc;
    const size_t cap = c->opt.reserved[2] > 0 ? (size_t)c->opt.reserved[2] << 20 : kBlockStageBytes;
    const int64_t chunk = std::max<int64_t>(1, (int64_t)(cap / (6 * ppb * sizeof(double))));
    const size_t need = (size_t)std::min<int64_t>(chunk, n) * 6 * ppb * sizeof(double);
    if (c->bstage_bytes < need) {
        CU(cudaStreamSynchronize(c->stream));
        CU(cudaStreamSynchronize(c->copy_stream));
        for (int b = 0; b < 2; ++b) {
            if (c->bstage[b]) CU(cudaFree(c->bstage[b]));
            c->bstage[b] = nullptr;
        }
        c->bstage_bytes = 0;
        for (int b = 0; b < 2; ++b) CU(cudaMalloc(&c->bstage[b], need));
        c->bstage_bytes = need;
    }
    IngestParams p = ingest_params(c);
    const int64_t end = step0 + n;
    int64_t s = step0;
    while (s < end) {
        // segment: up to and including the next closing call
        int64_t stop = end;
        auto itv = c->event_at.lower_bound(s);
        if (itv != c->event_at.end() && itv->first < end) stop = itv->first + 1;
        const int ev_idx = (itv != c->event_at.end() && itv->first == stop - 1) ? itv->second : -1;
        for (int b = 0; b < nblocks; ++b) {
            for (int64_t t = s; t < stop; t += chunk) {
                const int64_t m = std::min(chunk, stop - t);
                const int buf = c->stage_next;
                c->stage_next ^= 1;
                CU(cudaStreamWaitEvent(c->copy_stream, c->used_done[buf], 0));
                // one region per species: x then u, [m][3][count] each
                double* region = c->bstage[buf];
                for (int sp = 0; sp < S; ++sp) {
                    int64_t lo, cnt;
                    range(sp, b, lo, cnt);
                    if (cnt == 0) continue;
                    const int64_t g0 = c->in_off[sp] + lo;              // input column
                    double* sx = region;
                    double* su = sx + m * 3 * cnt;
                    region = su + m * 3 * cnt;
                    const double* xs = x + ((t - step0) * 3) * N + g0;
                    const double* us = u + ((t - step0) * 3) * N + g0;
                    CU(cudaMemcpy2DAsync(sx, cnt * sizeof(double), xs, N * sizeof(double),
                                         cnt * sizeof(double), (size_t)(m * 3),
                                         cudaMemcpyHostToDevice, c->copy_stream));
                    CU(cudaMemcpy2DAsync(su, cnt * sizeof(double), us, N * sizeof(double),
                                         cnt * sizeof(double), (size_t)(m * 3),
                                         cudaMemcpyHostToDevice, c->copy_stream));
                }
                CU(cudaEventRecord(c->copy_done[buf], c->copy_stream));
                CU(cudaStreamWaitEvent(c->stream, c->copy_done[buf], 0));
                region = c->bstage[buf];
                for (int sp = 0; sp < S; ++sp) {
                    int64_t lo, cnt;
                    range(sp, b, lo, cnt);
                    if (cnt == 0) continue;
                    const int64_t g0 = c->in_off[sp] + lo;
                    p.x = region;
                    p.u = region + m * 3 * cnt;
                    region += 2 * m * 3 * cnt;
                    p.step0 = t;
                    p.n_steps = (int32_t)m;
                    p.first = g0;
                    p.count = cnt;
                    p.ld = cnt;
                    p.xoff = g0;
                    rc = seg_scratch(c, cnt, m, p);
                    if (rc) return rc;
                    if (c->time_ingest)
                        CU(cudaEventRecord(next_event(c->ing_ev, c->ing_used, true), c->stream));
                    cudaError_t e = launch_ingest(p, c->stream);
                    if (e != cudaSuccess)
                        return fail(c, RAD_ECUDA, "ingest launch failed: %s", cudaGetErrorString(e));
                    if (c->time_ingest)
                        CU(cudaEventRecord(next_event(c->ing_ev, c->ing_used, false), c->stream));
                    ++c->ing_launches;
                }
                CU(cudaEventRecord(c->used_done[buf], c->stream));
            }
            if (ev_idx >= 0) {
                rc = launch_event(c, c->blk_events[ev_idx][b]);
                if (rc) return rc;
            }
        }
        s = stop;
    }
    // the caller may reuse its host buffers once this returns
    CU(cudaStreamSynchronize(c->copy_stream));
    return RAD_OK;
}

// Capture the launches of one step kind on a private stream, instantiate, and
// remember the ingest kernel node so that each call can patch its inputs in.
static int graph_for(rad_ctx* c, int kind, const IngestParams& ip, StepGraph** out)
{
    if ((int)c->graphs.size() < 1 + (int)c->events.size()) c->graphs.resize(1 + c->events.size());
    StepGraph& g = c->graphs[kind];
    if (!g.exec) {
        if (c->fault.graph)
            return fail(c, kGraphUnavailable, "step graph capture failed (RAD_FAULT=graph)");
        if (!c->cap_stream) CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_ingest(ip, c->cap_stream);
        if (e == cudaSuccess && kind > 0) {
            Event& ev = c->events[kind - 1];
            if (!ev.items.empty()) {
                const int grid = (int)std::min<int64_t>((int64_t)ev.items.size(), blocks_per_sm(c) * c->sms);
                Accum32Params p{};
                p.items = ev.d_items;
                p.n_items = (int32_t)ev.items.size();
                p.counter = c->d_counter;
                p.wins = c->d_wins;
                p.species = c->d_species;
                p.dirs32 = c->d_dirs32;
                p.omega = c->d_om32;
                p.nu_hi = c->d_nuhi;
                p.nu_lo = c->d_nulo;
                p.slab32 = c->slab32;
                p.anc32 = c->anc32;
                p.ring = c->ring;
                p.nblk = c->nblk;
                p.comps = c->comps;
                p.dt_hi = (float)(c->dt / c->nsub);
                p.dt_lo = (float)(c->dt / c->nsub - (double)p.dt_hi);
                p.acc = c->acc;
                p.err_word = c->d_err;
                e = cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->cap_stream);
                if (e == cudaSuccess && !accum32_dispatch(&p, c->cfg, grid, c->cap_stream, &e, nullptr))
                    e = cudaErrorInvalidValue;
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();   // capture errors are not sticky: clear the last error
            return fail(c, kGraphUnavailable, "step graph capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        g.graph = graph;
        size_t n = 0;
        CU(cudaGraphGetNodes(graph, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        CU(cudaGraphGetNodes(graph, nodes.data(), &n));
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            CU(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            CU(cudaGraphKernelNodeGetParams(nd, &kp));
            if (kp.func == ingest_kernel_ptr()) g.ingest_node = nd;
        }
        if (!g.ingest_node) return fail(c, RAD_ECUDA, "ingest node not found in the step graph");
        CU(cudaGraphInstantiate(&g.exec, graph, 0));
    }
    *out = &g;
    return RAD_OK;
}

// One step through its graph: patch the ingest node's parameters, replay.
static int step_via_graph(rad_ctx* c, int64_t step, const double* x, const double* u)
{
    IngestParams p = ingest_params(c);
    p.x = x;
    p.u = u;
    p.n_steps = 1;
    p.step0 = step;
    int kind = 0;
    if (!c->opt.defer) {
        auto itv = c->event_at.find(step);
        if (itv != c->event_at.end()) kind = 1 + itv->second;
    }
    StepGraph* g = nullptr;
    int rc = graph_for(c, kind, p, &g);
    if (rc) return rc;
    cudaKernelNodeParams kp;
    CU(cudaGraphKernelNodeGetParams(g->ingest_node, &kp));
    void* args[1] = {&p};
    kp.kernelParams = args;
    kp.extra = nullptr;
    CU(cudaGraphExecKernelNodeSetParams(g->exec, g->ingest_node, &kp));
    if (kind > 0) CU(cudaEventRecord(next_event(c->acc_ev, c->acc_used, true), c->stream));
    CU(cudaGraphLaunch(g->exec, c->stream));
    if (kind > 0) {
        CU(cudaEventRecord(next_event(c->acc_ev, c->acc_used, false), c->stream));
        ++c->acc_launches;
    }
    ++c->ing_launches;
    return RAD_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// Everything finalize and the partial-sum export share: every window's last
// sample must be in, deferred windows are evaluated (once), then `copy` enqueues
// the output; device-side error flags are checked after the stream drains.
template <class F>
static int complete_windows(rad_ctx* c, F copy)
{
    if (c->next_step < c->max_s1 + 1)
        return fail(c, RAD_EINCOMPLETE, "window needs step %lld, last step given is %lld",
                    (long long)c->max_s1, (long long)c->next_step - 1);
    int rc = freeze(c);
    if (rc) return rc;
    CU(cudaSetDevice(c->device));
    if (c->opt.defer && !c->deferred_done) {
        for (auto& ev : c->events) {
            rc = launch_event(c, ev);
            if (rc) return rc;
        }
        c->deferred_done = true;
    }
    rc = copy();
    if (rc) return rc;
    int errw = 0;
    CU(cudaMemcpyAsync(&errw, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (errw & kErrTimeout) return fail(c, RAD_ETIMEOUT, "a device-side wait expired");
    if (errw & kErrNaN) return fail(c, RAD_ENAN, "non-finite x or u in the input");
    return RAD_OK;
}

namespace rad {
cudaStream_t ctx_stream(const rad_ctx* c) { return c ? c->stream : nullptr; }
int64_t ctx_particles(const rad_ctx* c) { return c ? c->n_in : -1; }
int64_t ctx_next_step(const rad_ctx* c) { return c ? c->next_step : -1; }
}  // namespace rad

extern "C" {

int rad_init(rad_ctx** out, const double* dirs, int32_t D, const double* freqs,
             const int32_t* grid_len, int32_t n_grids, double dt, const rad_species* sp,
             int32_t n_species, const rad_window* win, int32_t n_win, int32_t mode,
             int32_t precision, double box_L, void* cuda_stream)
{
    if (!out) return RAD_EINVAL;
    *out = nullptr;
    if (!dirs || D < 1 || !freqs || !grid_len || n_grids < 1 || !(dt > 0.0) || !std::isfinite(dt) ||
        !sp || n_species < 1 || n_species > kMaxSpecies || !win || n_win < 1 ||
        (mode != RAD_INCOHERENT && mode != RAD_COHERENT) ||
        (precision != RAD_FP64 && precision != RAD_FP32_SPLIT) || !(box_L >= 0.0) ||
        !std::isfinite(box_L))
        return RAD_EINVAL;
    rad_ctx* c = new (std::nothrow) rad_ctx();
    if (!c) return RAD_ENOMEM;
    auto bail = [&](int rc) {
        rad_destroy(c);
        return rc;
    };
    if (!parse_fault_env(c->fault)) return bail(RAD_EINVAL);
    c->D = D;
    c->n_grids = n_grids;
    c->dt = dt;
    c->box_L = box_L;
    c->mode = mode;
    c->precision = precision;
    c->n_species = n_species;
    c->stream = (cudaStream_t)cuda_stream;
    int64_t nf = 0;
    for (int g = 0; g < n_grids; ++g) {
        if (grid_len[g] < 1) return bail(RAD_EINVAL);
        c->grid_off.push_back((int)nf);
        c->grid_len.push_back(grid_len[g]);
        nf += grid_len[g];
    }
    for (int64_t i = 0; i < nf; ++i)
        if (!std::isfinite(freqs[i])) return bail(RAD_EINVAL);
    c->h_freqs.assign(freqs, freqs + nf);
    c->in_off.push_back(0);
    int64_t col = 0;
    for (int s = 0; s < n_species; ++s) {
        if (sp[s].count < 0 || !std::isfinite(sp[s].charge)) return bail(RAD_EINVAL);
        c->species.push_back(sp[s]);
        c->col_off.push_back((int32_t)col);
        col += (sp[s].count + kTileP - 1) / kTileP * kTileP;
        c->in_off.push_back(c->in_off.back() + sp[s].count);
    }
    c->n_in = c->in_off.back();
    c->ncols = std::max<int64_t>(col, kTileP);
    if (c->ncols > (int64_t)1 << 30) return bail(RAD_EINVAL);
    int64_t min_s0 = INT64_MAX;
    for (int w = 0; w < n_win; ++w) {
        const rad_window& W = win[w];
        if (W.s0 < 0 || W.s1 < W.s0 || W.freq_grid < 0 || W.freq_grid >= n_grids ||
            (n_species < 32 && (W.species_mask >> n_species) != 0) || W.reserved != 0 ||
            (W.dir_set && W.n_dir_set < 1))
            return bail(RAD_EINVAL);
        std::vector<int32_t> wd;
        if (W.dir_set) {
            for (int32_t i = 0; i < W.n_dir_set; ++i) {
                if (W.dir_set[i] < 0 || W.dir_set[i] >= D) return bail(RAD_EINVAL);
                wd.push_back(W.dir_set[i]);
            }
        } else {
            for (int32_t d = 0; d < D; ++d) wd.push_back(d);
        }
        rad_window Wc = W;
        Wc.dir_set = nullptr;                 // the caller's array is not kept
        Wc.n_dir_set = (int32_t)wd.size();
        c->wins.push_back(Wc);
        c->out_off.push_back(c->out_len);
        c->out_len += (int64_t)wd.size() * grid_len[W.freq_grid];
        c->win_dirs.push_back(std::move(wd));
        c->max_s1 = std::max<int64_t>(c->max_s1, W.s1);
        min_s0 = std::min<int64_t>(min_s0, W.s0);
    }
    // ring length: longest window (eager) or the whole span (defer is decided
    // later, so size for the span; the ring is what the windows need at once)
    int64_t span = std::max<int64_t>(1, c->max_s1 - min_s0);
    c->ring = (span + 31) / 32 * 32 + 64;

    int rc;
    {
        int dev;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return bail(fail(c, RAD_ECUDA, "no CUDA device: %s", cudaGetErrorString(e)));
        c->device = dev;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return bail(RAD_ECUDA);
        c->sms = prop.multiProcessorCount;
    }
    (void)rc;
#define CUB(call)                                                      \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess)                                         \
            return bail(e_ == cudaErrorMemoryAllocation ? RAD_ENOMEM : RAD_ECUDA); \
    } while (0)
    // directions and bases
    std::vector<float> d32((size_t)D * 12);
    std::vector<double> d64((size_t)D * 9);
    for (int d = 0; d < D; ++d) {
        double n[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
        double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(l > 0.0) || !std::isfinite(l)) return bail(RAD_EINVAL);
        for (int i = 0; i < 3; ++i) n[i] /= l;
        double e1[3], e2[3];
        basis(n, e1, e2);
        for (int i = 0; i < 3; ++i) {
            d32[12 * d + i] = (float)n[i];
            d32[12 * d + 3 + i] = (float)e1[i];
            d32[12 * d + 6 + i] = (float)e2[i];
            d32[12 * d + 9 + i] = (float)(n[i] - (double)(float)n[i]);
            d64[9 * d + i] = n[i];
            d64[9 * d + 3 + i] = e1[i];
            d64[9 * d + 6 + i] = e2[i];
        }
    }
    std::vector<float> om32(nf), nuh(nf), nul(nf);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < nf; ++i) {
        om32[i] = (float)freqs[i];
        const double nu = freqs[i] / two_pi;
        nuh[i] = (float)nu;
        nul[i] = (float)(nu - (double)nuh[i]);
    }
    std::vector<WinDev> wd(n_win);
    for (int w = 0; w < n_win; ++w) {
        wd[w].s0 = win[w].s0;
        wd[w].s1 = win[w].s1;
        wd[w].grid_off = c->grid_off[win[w].freq_grid];
        wd[w].grid_len = c->grid_len[win[w].freq_grid];
        wd[w].out_off = c->out_off[w];
        wd[w].sel = -1;
    }
    c->win_sel.assign(n_win, -1);
    std::vector<SpeciesDev> sd(n_species);
    for (int s = 0; s < n_species; ++s) {
        sd[s].qdt = sp[s].charge * dt;
        sd[s].col0 = c->col_off[s];
        sd[s].count = (int32_t)sp[s].count;
    }
    CUB(cudaMalloc(&c->d_dirs32, d32.size() * sizeof(float)));
    CUB(cudaMalloc(&c->d_dirs64, d64.size() * sizeof(double)));
    CUB(cudaMalloc(&c->d_om32, nf * sizeof(float)));
    CUB(cudaMalloc(&c->d_nuhi, nf * sizeof(float)));
    CUB(cudaMalloc(&c->d_nulo, nf * sizeof(float)));
    CUB(cudaMalloc(&c->d_om64, nf * sizeof(double)));
    CUB(cudaMalloc(&c->d_wins, n_win * sizeof(WinDev)));
    CUB(cudaMalloc(&c->d_sel, kMaxSelectors * sizeof(SelectorDev)));
    CUB(cudaMalloc(&c->d_species, n_species * sizeof(SpeciesDev)));
    CUB(cudaMemcpy(c->d_dirs32, d32.data(), d32.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_dirs64, d64.data(), d64.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_om32, om32.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_nuhi, nuh.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_nulo, nul.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_om64, freqs, nf * sizeof(double), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_wins, wd.data(), n_win * sizeof(WinDev), cudaMemcpyHostToDevice));
    CUB(cudaMemcpy(c->d_species, sd.data(), n_species * sizeof(SpeciesDev), cudaMemcpyHostToDevice));

    // ring and state
    if (c->fault.alloc) return bail(RAD_ENOMEM);
    const int64_t nc = c->ncols;
    if (precision == RAD_FP64) {
        CUB(cudaMalloc(&c->slab64, (size_t)c->ring * c->comps * nc * sizeof(double)));
        CUB(cudaMemset(c->slab64, 0, (size_t)c->ring * c->comps * nc * sizeof(double)));
    } else {
        CUB(cudaMalloc(&c->slab32, (size_t)c->ring * c->comps * nc * sizeof(float)));
        CUB(cudaMemset(c->slab32, 0, (size_t)c->ring * c->comps * nc * sizeof(float)));
    }
    CUB(cudaMalloc(&c->x_prev, 3 * nc * sizeof(double)));
    CUB(cudaMalloc(&c->r_prev, 3 * nc * sizeof(double)));
    CUB(cudaMalloc(&c->u_prev, 3 * nc * sizeof(double)));
    const size_t acc_n = (size_t)c->out_len * (mode == RAD_COHERENT ? 4 : 1);
    CUB(cudaMalloc(&c->acc, std::max<size_t>(1, acc_n) * sizeof(double)));
    CUB(cudaMemset(c->acc, 0, std::max<size_t>(1, acc_n) * sizeof(double)));
    CUB(cudaMalloc(&c->d_out, std::max<int64_t>(1, c->out_len) * sizeof(double)));
    CUB(cudaMalloc(&c->d_err, sizeof(int)));
    CUB(cudaMalloc(&c->d_counter, sizeof(int)));
    CUB(cudaMemset(c->d_err, 0, sizeof(int)));
    CUB(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        CUB(cudaEventCreateWithFlags(&c->copy_done[b], cudaEventDisableTiming));
        CUB(cudaEventCreateWithFlags(&c->used_done[b], cudaEventDisableTiming));
    }
    CUB(cudaDeviceSynchronize());
#undef CUB
    *out = c;
    return RAD_OK;
}

int rad_set_options(rad_ctx* c, const rad_options* o)
{
    if (!c || !o) return RAD_EINVAL;
    if (c->frozen) return fail(c, RAD_ESTATE, "options must be set before the first step");
    if (o->variant < 0 || o->variant > 3) return fail(c, RAD_EINVAL, "variant out of range");
    if (o->variant == RAD_VARIANT_PRECISE &&
        ((o->anchor_K != 0 && o->anchor_K != 32) || (o->freq_per_lane != 0 && o->freq_per_lane != 8) ||
         o->blocks_per_sm == 4))
        return fail(c, RAD_EINVAL,
                    "the precise-phase variant is built for anchor_K 32, 8 frequencies per thread, "
                    "2 or 3 blocks per SM");
    if (o->anchor_K != 0 && o->anchor_K != 8 && o->anchor_K != 16 && o->anchor_K != 32)
        return fail(c, RAD_EINVAL, "anchor_K must be 0, 8, 16 or 32");
    if (o->freq_per_lane != 0 && o->freq_per_lane != 4 && o->freq_per_lane != 8 &&
        o->freq_per_lane != 16)
        return fail(c, RAD_EINVAL, "freq_per_lane must be 0, 4, 8 or 16");
    if (o->reserved[3] < 0) return fail(c, RAD_EINVAL, "phase budget must be >= 0");
    if (o->subcycle < 0 || o->subcycle > 64)
        return fail(c, RAD_EINVAL, "subcycle must be in [0, 64]");
    if (o->blocks_per_sm != 0 && o->blocks_per_sm != 2 && o->blocks_per_sm != 3 &&
        o->blocks_per_sm != 4)
        return fail(c, RAD_EINVAL, "blocks_per_sm must be 0, 2, 3 or 4");
    c->opt = *o;
    c->time_ingest = o->reserved[0] != 0;
    return RAD_OK;
}

int rad_set_selectors(rad_ctx* c, const rad_selector* sel, int32_t n_sel,
                      const int32_t* window_selector)
{
    if (!c) return RAD_EINVAL;
    if (c->frozen) return fail(c, RAD_ESTATE, "selectors must be set before the first step");
    if (n_sel < 0 || n_sel > kMaxSelectors || (n_sel > 0 && !sel) || !window_selector)
        return fail(c, RAD_EINVAL, "bad selector arguments");
    std::vector<SelectorDev> h(n_sel);
    for (int i = 0; i < n_sel; ++i) {
        const rad_selector& S = sel[i];
        SelectorDev& d = h[i];
        d = SelectorDev{};
        d.kind = S.kind;
        if (S.kind == RAD_SEL_BOX) {
            for (int q = 0; q < 3; ++q) {
                if (!std::isfinite(S.lo[q]) || !std::isfinite(S.hi[q]))
                    return fail(c, RAD_EINVAL, "selector %d: non-finite box", i);
                d.lo[q] = S.lo[q];
                d.hi[q] = S.hi[q];
            }
        } else if (S.kind == RAD_SEL_CONE) {
            const double l = std::sqrt(S.axis[0] * S.axis[0] + S.axis[1] * S.axis[1] +
                                       S.axis[2] * S.axis[2]);
            if (!(l > 0.0) || !std::isfinite(l) || !(S.dtheta >= 0.0) || !std::isfinite(S.theta_c))
                return fail(c, RAD_EINVAL, "selector %d: bad cone", i);
            for (int q = 0; q < 3; ++q) d.axis[q] = S.axis[q] / l;
            const double a_hi = std::min(M_PI, S.theta_c + S.dtheta);
            const double a_lo = std::max(0.0, S.theta_c - S.dtheta);
            d.cos_lo = std::cos(a_hi);
            d.cos_hi = std::cos(a_lo);
        } else {
            return fail(c, RAD_EINVAL, "selector %d: unknown kind %d", i, S.kind);
        }
    }
    for (size_t w = 0; w < c->wins.size(); ++w)
        if (window_selector[w] < -1 || window_selector[w] >= n_sel)
            return fail(c, RAD_EINVAL, "window %zu: selector index out of range", w);
    CU(cudaSetDevice(c->device));
    if (n_sel > 0 && c->comps == kCompsPlain) {
        // the samples now carry their selector bits: the ring gains the flags word
        const size_t es = c->precision == RAD_FP64 ? sizeof(double) : sizeof(float);
        void*& slab = c->precision == RAD_FP64 ? reinterpret_cast<void*&>(c->slab64)
                                               : reinterpret_cast<void*&>(c->slab32);
        CU(cudaStreamSynchronize(c->stream));
        CU(cudaFree(slab));
        slab = nullptr;
        const size_t bytes = (size_t)c->ring * kComps * c->ncols * es;
        CU(cudaMalloc(&slab, bytes));
        CU(cudaMemset(slab, 0, bytes));
        c->comps = kComps;
    }
    if (n_sel > 0)
        CU(cudaMemcpy(c->d_sel, h.data(), n_sel * sizeof(SelectorDev), cudaMemcpyHostToDevice));
    c->n_sel = n_sel;
    c->win_sel.assign(window_selector, window_selector + c->wins.size());
    std::vector<WinDev> wd(c->wins.size());
    CU(cudaMemcpy(wd.data(), c->d_wins, wd.size() * sizeof(WinDev), cudaMemcpyDeviceToHost));
    for (size_t w = 0; w < wd.size(); ++w) wd[w].sel = c->win_sel[w];
    CU(cudaMemcpy(c->d_wins, wd.data(), wd.size() * sizeof(WinDev), cudaMemcpyHostToDevice));
    return RAD_OK;
}

int rad_get_options(const rad_ctx* c, rad_options* o)
{
    if (!c || !o) return RAD_EINVAL;
    *o = c->opt;
    if (c->graph_off) o->use_graph = 0;
    if (c->frozen && c->precision == RAD_FP32_SPLIT) {
        o->anchor_K = c->cfg.K;
        o->freq_per_lane = c->cfg.ft;
        o->blocks_per_sm = c->cfg.mb;
        o->variant = c->cfg.pm ? RAD_VARIANT_PRECISE
                                 : (c->cfg.np > 0 ? RAD_VARIANT_MIX : RAD_VARIANT_SFU);
        o->reserved[1] = c->cfg.np;
    }
    return RAD_OK;
}

int rad_accumulate_steps(rad_ctx* c, int64_t step0, int64_t n, const double* x, const double* u)
{
    if (!c) return RAD_EINVAL;
    if (n < 0 || (n > 0 && (!x || !u))) return fail(c, RAD_EINVAL, "bad step count or null input");
    if (step0 != c->next_step)
        return fail(c, RAD_ESTEP, "step %lld given, %lld expected", (long long)step0,
                    (long long)c->next_step);
    if (n == 0) return RAD_OK;
    if (c->fault.drop_step == step0) {   // test hook: this hand-over is lost once
        c->fault.drop_step = -1;
        return RAD_OK;
    }
    int rc = freeze(c);
    if (rc) return rc;
    CU(cudaSetDevice(c->device));
    const bool dx = is_device_ptr(x), du = is_device_ptr(u);
    if (dx && du && n == 1 && c->opt.use_graph && !c->graph_off &&
        c->precision == RAD_FP32_SPLIT) {
        rc = step_via_graph(c, step0, x, u);
        if (rc == kGraphUnavailable) {
            c->graph_off = true;   // direct launches from now on
            rc = ingest_device(c, step0, n, x, u);
        }
        if (rc) return rc;
    } else if (dx && du) {
        rc = ingest_device(c, step0, n, x, u);
        if (rc) return rc;
    } else if (!dx && !du && !c->opt.defer && n >= 64 && c->n_in >= 64 * kTileP * kHostBlocks) {
        rc = ingest_host_blocked(c, step0, n, x, u);
        if (rc) return rc;
    } else {
        // host inputs: double-buffered staging on a copy stream
        const int64_t per = 3 * c->n_in;
        int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, 64));
        if (c->stage_steps < chunk) {
            for (int b = 0; b < 2; ++b) {
                if (c->stage[b]) {
                    CU(cudaStreamSynchronize(c->stream));
                    CU(cudaFree(c->stage[b]));
                    c->stage[b] = nullptr;
                }
                CU(cudaMalloc(&c->stage[b], (size_t)std::max<int64_t>(1, 2 * chunk * per) * sizeof(double)));
            }
            c->stage_steps = chunk;
        }
        for (int64_t s = 0; s < n; s += chunk) {
            const int64_t m = std::min(chunk, n - s);
            const int b = c->stage_next;
            c->stage_next ^= 1;
            double* sx = c->stage[b];
            double* su = c->stage[b] + c->stage_steps * per;
            CU(cudaStreamWaitEvent(c->copy_stream, c->used_done[b], 0));
            const size_t bytes = (size_t)m * per * sizeof(double);
            if (dx) CU(cudaMemcpyAsync(sx, x + s * per, bytes, cudaMemcpyDeviceToDevice, c->copy_stream));
            else CU(cudaMemcpyAsync(sx, x + s * per, bytes, cudaMemcpyHostToDevice, c->copy_stream));
            if (du) CU(cudaMemcpyAsync(su, u + s * per, bytes, cudaMemcpyDeviceToDevice, c->copy_stream));
            else CU(cudaMemcpyAsync(su, u + s * per, bytes, cudaMemcpyHostToDevice, c->copy_stream));
            CU(cudaEventRecord(c->copy_done[b], c->copy_stream));
            CU(cudaStreamWaitEvent(c->stream, c->copy_done[b], 0));
            rc = ingest_device(c, step0 + s, m, sx, su);
            if (rc) return rc;
            CU(cudaEventRecord(c->used_done[b], c->stream));
        }
        // the caller may reuse its host buffers once this returns
        CU(cudaStreamSynchronize(c->copy_stream));
    }
    c->next_step = step0 + n;
    return RAD_OK;
}

int rad_accumulate(rad_ctx* c, int64_t step, const double* x, const double* u)
{
    return rad_accumulate_steps(c, step, 1, x, u);
}

int rad_finalize(rad_ctx* c, double* spectrum)
{
    if (!c) return RAD_EINVAL;
    if (!spectrum && c->out_len > 0) return fail(c, RAD_EINVAL, "null spectrum buffer");
    return complete_windows(c, [&]() -> int {
        if (c->out_len > 0) {
            finalize_kernel<<<(unsigned)std::min<int64_t>((c->out_len + 255) / 256, 4096), 256, 0,
                              c->stream>>>(c->acc, c->d_out, c->out_len, c->mode == RAD_COHERENT);
            CU(cudaGetLastError());
            const bool dev = is_device_ptr(spectrum);
            CU(cudaMemcpyAsync(spectrum, c->d_out, c->out_len * sizeof(double),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        }
        return RAD_OK;
    });
}

int rad_partial_sums(rad_ctx* c, double* out)
{
    if (!c) return RAD_EINVAL;
    if (!out && c->out_len > 0) return fail(c, RAD_EINVAL, "null output buffer");
    return complete_windows(c, [&]() -> int {
        const size_t n = (size_t)c->out_len * (c->mode == RAD_COHERENT ? 4 : 1);
        if (n > 0) {
            const bool dev = is_device_ptr(out);
            CU(cudaMemcpyAsync(out, c->acc, n * sizeof(double),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        }
        return RAD_OK;
    });
}

int rad_spectrum_from_sums(const double* sums, int64_t n_bins, int32_t mode, double* spectrum,
                           void* cuda_stream)
{
    if (n_bins < 0 || (mode != RAD_INCOHERENT && mode != RAD_COHERENT)) return RAD_EINVAL;
    if (n_bins == 0) return RAD_OK;
    if (!sums || !spectrum || !current_device_ptr(sums) || !current_device_ptr(spectrum))
        return RAD_EINVAL;
    finalize_kernel<<<(unsigned)std::min<int64_t>((n_bins + 255) / 256, 4096), 256, 0,
                      (cudaStream_t)cuda_stream>>>(sums, spectrum, n_bins, mode == RAD_COHERENT);
    return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_next_shard(rad_ctx* c)
{
    if (!c) return RAD_EINVAL;
    if (c->next_step < c->max_s1 + 1)
        return fail(c, RAD_EINCOMPLETE, "window needs step %lld, last step given is %lld",
                    (long long)c->max_s1, (long long)c->next_step - 1);
    int rc = freeze(c);
    if (rc) return rc;
    CU(cudaSetDevice(c->device));
    if (c->opt.defer && !c->deferred_done) {
        for (auto& ev : c->events) {
            rc = launch_event(c, ev);
            if (rc) return rc;
        }
    }
    // the ring, anchors and per-particle ingest state are rewritten from step 0
    // by the next shard's calls; the accumulators keep their sums
    c->next_step = 0;
    c->deferred_done = false;
    return RAD_OK;
}

int rad_reset(rad_ctx* c)
{
    if (!c) return RAD_EINVAL;
    CU(cudaSetDevice(c->device));
    const size_t acc_n = (size_t)c->out_len * (c->mode == RAD_COHERENT ? 4 : 1);
    CU(cudaMemsetAsync(c->acc, 0, std::max<size_t>(1, acc_n) * sizeof(double), c->stream));
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    c->next_step = 0;
    c->deferred_done = false;
    return RAD_OK;
}

int64_t rad_spectrum_size(const rad_ctx* c) { return c ? c->out_len : -1; }

int64_t rad_updates(const rad_ctx* c)
{
    if (!c) return -1;
    int64_t tot = 0;
    for (const auto& W : c->wins) {
        int64_t np = 0;
        for (int s = 0; s < c->n_species; ++s)
            if ((W.species_mask >> s) & 1u) np += c->species[s].count;
        tot += np * (W.s1 - W.s0) * W.n_dir_set * c->grid_len[W.freq_grid];
    }
    return tot * c->nsub;
}

int rad_timing(rad_ctx* c, double* accum_ms, double* ingest_ms, int64_t* accum_launches,
               int64_t* ingest_launches)
{
    if (!c) return RAD_EINVAL;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    double a = 0, g = 0;
    for (size_t i = 0; i < c->acc_used; ++i) {
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, c->acc_ev[i].first, c->acc_ev[i].second));
        a += ms;
    }
    for (size_t i = 0; i < c->ing_used; ++i) {
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, c->ing_ev[i].first, c->ing_ev[i].second));
        g += ms;
    }
    if (accum_ms) *accum_ms = a;
    if (ingest_ms) *ingest_ms = g;
    if (accum_launches) *accum_launches = c->acc_launches;
    if (ingest_launches) *ingest_launches = c->ing_launches;
    return RAD_OK;
}

const char* rad_last_error(const rad_ctx* c)
{
    if (!c) return kNoCtx;
    return c->err.c_str();
}

void rad_destroy(rad_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& ev : c->events) cudaFree(ev.d_items);
    for (auto& row : c->blk_events)
        for (auto& ev : row) cudaFree(ev.d_items);
    void* bufs[] = {c->slab32, c->slab64, c->anc32, c->x_prev, c->r_prev, c->u_prev,
                    c->d_dirs32, c->d_dirs64, c->d_om32, c->d_nuhi, c->d_nulo,
                    c->d_om64, c->d_wins, c->d_sel, c->d_species, c->acc, c->d_out, c->d_err, c->d_counter,
                    c->stage[0], c->stage[1], c->bstage[0], c->bstage[1], c->seg_buf};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (auto& pr : c->acc_ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& pr : c->ing_ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->copy_done[b]) cudaEventDestroy(c->copy_done[b]);
        if (c->used_done[b]) cudaEventDestroy(c->used_done[b]);
    }
    for (auto& g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    delete c;
}

}  // extern "C"
