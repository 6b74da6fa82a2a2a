// Host side of libbude.so: the C ABI declared in include/bude.h.
//
// Decks own repacked device copies of their inputs and a growable scratch
// workspace (cross-CTA partial sums and arrival tickets of the persistent
// kernel).  Launch planning -- the flat work space, the persistent grid and
// the shared-memory carve-up -- happens here; all arithmetic of the path runs
// in the kernels.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bude_internal.h"

using namespace bude;

namespace {
// Allocations left before the injected failure; 0 = no injection.
std::atomic<int> g_fail_alloc_in{0};
}  // namespace

namespace bude {

cudaError_t dev_alloc(void** p, size_t bytes)
{
    int k = g_fail_alloc_in.load();
    while (k > 0 && !g_fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

Range::Range(const char* name) { nvtxRangePushA(name); }
Range::~Range() { nvtxRangePop(); }

}  // namespace bude

struct bude_deck {
    int device = 0;
    int n_lig = 0, n_pro = 0, n_types = 0, n_rows = 0;
    float4* pro = nullptr;   // [n_pro] sorted by type, coordinates as given (FP64 kernel)
    float4* pro_c = nullptr; // [n_pro] the same atoms in the frame centred on centre[] (FP32 kernels)
    float centre[3] = {0.f, 0.f, 0.f};  // midpoint of the protein's bounding box
    float4* lig = nullptr;   // [n_lig] row-mapped
    PairF* tabF = nullptr;   // [n_rows][n_types]
    PairG* tabG = nullptr;
    PairD* tabD = nullptr;
    int* row_type = nullptr; // [n_rows]
    float4* ff = nullptr;    // [n_types] forcefield rows as given
    // ligand and protein atoms of a polar type (hbtype != 0): a pair has a
    // desolvation term exactly when one of its atoms is polar
    int lig_polar = 0, pro_polar = 0;
    // scratch workspace of the plain and adjoint calls
    double* partial = nullptr;
    size_t partial_bytes = 0;
    unsigned* counter = nullptr;
    size_t counter_count = 0;
    // staging of bude_energies_host: poses [6][n] then energies [n]
    float* io = nullptr;
    size_t io_floats = 0;
};

namespace {

thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;

std::mutex g_opt_mutex;
bude_options g_default[4] = {
    {BUDE_FP32_IEEE, 8, 256, 0, 1, 0},
    {BUDE_FP32_FAST, 8, 256, 0, 1, 0},
    {BUDE_FP32_COMP, 8, 256, 0, 1, 0},
    {BUDE_FP64, 2, 256, 0, 1, 0},
};

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(BUDE_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(BUDE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DeviceInfo {
    int sms = 0;
    size_t smem_optin = 0;   // max dynamic + static per block
    size_t smem_per_sm = 0;
    size_t reserved_per_block = 0;
};

DeviceInfo device_info(int dev)
{
    static std::mutex m;
    static std::map<int, DeviceInfo> cache;
    std::lock_guard<std::mutex> lk(m);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceInfo d;
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    d.smem_optin = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    d.smem_per_sm = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    d.reserved_per_block = (size_t)v;
    cache[dev] = d;
    return d;
}

const void* kernel_for(int variant, int P, bool G, bool cull = false)
{
    // cutoff culling is built for the packed FP32 kernels (even P); elsewhere
    // the flag is ignored (the results are the same either way)
    if (cull && P % 2 == 0) {
        switch (variant) {
        case BUDE_FP32_IEEE: return kernel_ieee_cull(P, G);
        case BUDE_FP32_FAST: return kernel_fast_cull(P, G);
        case BUDE_FP32_COMP: return kernel_comp_cull(P, G);
        }
    }
    switch (variant) {
    case BUDE_FP32_IEEE: return kernel_ieee(P, G);
    case BUDE_FP32_FAST: return kernel_fast(P, G);
    case BUDE_FP32_COMP: return kernel_comp(P, G);
    case BUDE_FP64: return kernel_f64(P, G);
    }
    return nullptr;
}

// Packed FP32x2 kernels: FP32 variants with an even P (mirrors the kernel).
bool packed(int variant, int P, bool G)
{
    (void)G;
    return variant != BUDE_FP64 && P % 2 == 0;
}

// Bytes of one type-pair record in shared memory for a variant / mode.
size_t record_bytes(int variant, bool G, int P)
{
    if (variant == BUDE_FP64) return sizeof(PairD);
    if (packed(variant, P, G)) return G ? 96 : 64;
    return G ? sizeof(PairG) : sizeof(PairF);
}

// Bytes of one staged protein atom in shared memory (mirrors PRO4).
size_t protein_bytes(int variant, int P, bool G)
{
    return (packed(variant, P, G) || variant == BUDE_FP64) ? 32 : 16;
}

// Per-chunk run table and ligand-row cost prefix of the packed kernels.
size_t run_bytes(int variant, int P, bool G, int n_types, int n_lig)
{
    // the packed kernels and the FP64 kernel walk same-type runs (mirrors RUNS)
    return (packed(variant, P, G) || variant == BUDE_FP64) ? run_area_bytes(n_types, n_lig) : 0;
}

// Dynamic shared memory of pose_kernel before the pair table and protein
// chunk: max(transforms, warp partials) + final sums.  Mirrors the kernel.
size_t smem_fixed(int variant, int P, bool G, int block)
{
    const size_t TP = 32u * (size_t)P;
    const size_t W = (size_t)block / 32;
    const size_t treal = variant == BUDE_FP64 ? 8 : 4;
    const size_t tacc = (variant == BUDE_FP64 || variant == BUDE_FP32_COMP) ? 8 : 4;
    size_t regA = std::max(12 * TP * treal, W * TP * tacc);
    regA = (regA + 15) & ~size_t(15);
    const size_t NV = G ? 7 : 1;
    return regA + NV * TP * 8;
}

// Static shared memory of the kernel (Instance + flag), rounded up.
constexpr size_t kStaticSmem = 256;
static_assert(sizeof(Instance) + sizeof(int) <= kStaticSmem, "static shared memory of pose_kernel");

struct Resolved {
    int variant, P, block, tile, cps, cull;
};

int resolve_options(const bude_options* o, bool G, Resolved* r)
{
    int variant = o ? o->variant : BUDE_FP32_IEEE;
    if (variant < 0 || variant > 3) return fail(BUDE_ERR_INVALID_ARG, "unknown variant %d", variant);
    bude_options d;
    {
        std::lock_guard<std::mutex> lk(g_opt_mutex);
        d = g_default[variant];
    }
    r->variant = variant;
    r->P = (o && o->ppwi) ? o->ppwi : d.ppwi;
    r->block = (o && o->block) ? o->block : d.block;
    r->tile = (o && o->tile) ? o->tile : d.tile;
    r->cps = (o && o->ctas_per_sm) ? o->ctas_per_sm : d.ctas_per_sm;
    r->cull = (o && o->cull) ? o->cull : d.cull;
    if (r->cull != 0 && r->cull != 1) return fail(BUDE_ERR_INVALID_ARG, "cull %d: need 0 or 1", r->cull);
    if (G && variant != BUDE_FP64 && r->P > 8) r->P = 8;
    if (G && variant == BUDE_FP64 && r->P > 4) r->P = 4;
    if (r->block < 64 || r->block > 1024 || r->block % 32)
        return fail(BUDE_ERR_INVALID_ARG, "block %d: need a multiple of 32 in [64, 1024]", r->block);
    if (r->tile < 0) return fail(BUDE_ERR_INVALID_ARG, "tile %d < 0", r->tile);
    if (r->cps < 1 || r->cps > 32) return fail(BUDE_ERR_INVALID_ARG, "ctas_per_sm %d", r->cps);
    const void* fn = kernel_for(variant, r->P, G);
    if (!fn)
        return fail(BUDE_ERR_UNSUPPORTED, "poses per thread %d not built for variant %d%s", r->P,
                    variant, G ? " (adjoint)" : "");
    // The defaults are one shape per variant, usually the energy kernel's; an
    // adjoint call that takes its block from them gets at most as many
    // threads as the adjoint kernel's registers let one CTA have (an explicit
    // block is left as asked, and fails at launch if it cannot be resident).
    if (G && !(o && o->block)) {
        const void* fk = r->cull ? kernel_for(variant, r->P, G, true) : nullptr;
        if (!fk) fk = fn;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fk) == cudaSuccess) {
            const int cap = fa.maxThreadsPerBlock / 32 * 32;
            if (cap >= 64 && r->block > cap) r->block = cap;
        }
    }
    return BUDE_OK;
}

// Shared memory one CTA may use when cps CTAs share an SM.
size_t smem_budget(const DeviceInfo& di, int cps)
{
    size_t per = di.smem_per_sm / (size_t)cps;
    per = per > di.reserved_per_block ? per - di.reserved_per_block : 0;
    return std::min(per, di.smem_optin) - kStaticSmem;
}

struct InstanceShape {
    int n_lig, n_pro, n_types, n_rows;
    long long n_poses;
};

// Protein chunk length for one instance, or -1 when even the table does not fit.
int chunk_for(const InstanceShape& s, const Resolved& r, bool G, size_t budget)
{
    const size_t fixed = smem_fixed(r.variant, r.P, G, r.block);
    const size_t table = (size_t)s.n_rows * s.n_types * record_bytes(r.variant, G, r.P) +
                         run_bytes(r.variant, r.P, G, s.n_types, s.n_lig);
    const size_t pb = protein_bytes(r.variant, r.P, G);
    if (fixed + table + pb * 32 > budget) return -1;
    size_t cap = (budget - fixed - table) / pb;
    int want = s.n_pro;
    if (r.tile > 0) want = std::min(want, r.tile);
    int ch = (int)std::min<size_t>((size_t)std::max(want, 1), cap);
    return std::max(ch, 1);
}

// The CTAs a launch over instances inst (their units' costs w, total cost
// u_total) may use, given at most `grid`.  A launch of several instances
// splits their cost evenly over the CTAs, and a CTA's range holds at least
// one unit only if its share of the cost is at least the dearest unit's: a
// CTA without units inside a tile would be counted among the tile's
// arrivals and never arrive, leaving the tile unwritten.  So the grid is
// capped at u_total / (dearest unit).  One instance splits by unit count,
// and grid <= units suffices.
long long split_grid(const std::vector<Instance>& inst, long long u_total, long long grid)
{
    grid = std::max(1ll, grid);
    if (inst.size() > 1 && u_total > 0) {
        long long wmax = 1;
        for (const Instance& J : inst) wmax = std::max<long long>(wmax, J.w);
        grid = std::max(1ll, std::min(grid, u_total / wmax));
    }
    return grid;
}

// Raise a kernel's limit on dynamic shared memory to at least `bytes`, never
// lower it.  The limit belongs to the function (per device), not to a launch:
// a lower value set for one call would fail a launch of another thread, or a
// replay of a captured graph, that needs more.  The limit only permits; each
// launch still asks for its own amount.
cudaError_t raise_smem_limit(const void* fn, size_t bytes)
{
    static std::mutex m;
    static auto& limits = *new std::map<std::pair<int, const void*>, size_t>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(m);
    size_t& cur = limits[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

struct Plan {
    std::vector<Instance> inst;
    long long n_total = 0;
    long long u_total = 0;  // cost of the flat space (the CTAs split it by cost)
    long long n_tiles = 0;
    size_t smem = 0;
    int grid = 0;
    const void* fn = nullptr;
};

// Build the launch of a set of instances; instances without work are left
// out (the caller zero-fills their outputs).
int make_plan(const std::vector<const bude_deck*>& decks, const std::vector<const float*>& poses,
              const std::vector<long long>& n, const std::vector<float*>& out,
              const std::vector<float*>& grad, const Resolved& r, bool G, int dev, Plan* pl)
{
    const DeviceInfo di = device_info(dev);
    const size_t budget = smem_budget(di, r.cps);
    const long long TP = 32ll * r.P;
    pl->inst.clear();
    long long k = 0, tiles = 0, u = 0;
    size_t smem_max = 0;
    for (size_t i = 0; i < decks.size(); ++i) {
        const bude_deck* d = decks[i];
        const long long K = (long long)d->n_lig * d->n_pro;
        if (n[i] == 0 || K == 0) continue;
        InstanceShape s{d->n_lig, d->n_pro, d->n_types, d->n_rows, n[i]};
        const int ch = chunk_for(s, r, G, budget);
        if (ch < 1)
            return fail(BUDE_ERR_UNSUPPORTED,
                        "type-pair table of %d x %d does not fit in shared memory", d->n_rows,
                        d->n_types);
        Instance I;
        memset(&I, 0, sizeof I);
        // FP32 kernels: the recentred copy, with the origin subtracted from
        // the translations; FP64: the atoms as given (exact in double)
        const bool f64 = r.variant == BUDE_FP64;
        I.pro = f64 ? d->pro : d->pro_c;
        I.ox = f64 ? 0.f : d->centre[0];
        I.oy = f64 ? 0.f : d->centre[1];
        I.oz = f64 ? 0.f : d->centre[2];
        I.lig = d->lig;
        // packed kernels stage their records from the adjoint table, which
        // also holds the steric factors sqrt|H|/R and sqrt|H|
        I.pair = r.variant == BUDE_FP64 ? (const void*)d->tabD
                 : (G || packed(r.variant, r.P, G)) ? (const void*)d->tabG
                                                    : (const void*)d->tabF;
        I.poses = poses[i];
        I.out = out[i];
        I.grad = G ? grad[i] : nullptr;
        I.n_poses = n[i];
        const long long nt = (n[i] + TP - 1) / TP;
        I.k_begin = k;
        I.k_end = k + nt * K;
        I.tile_begin = tiles;
        I.n_lig = d->n_lig;
        I.n_pro = d->n_pro;
        I.n_types = d->n_types;
        I.n_rows = d->n_rows;
        I.chunk = ch;
        // cost of one pair iteration, in tenths of the kernels' cost units: 10
        // for every pair plus 4 where the pair has a desolvation term (one of
        // its atoms polar), averaged over the deck's pairs
        {
            const double lp = d->lig_polar, pp = d->pro_polar;
            const double f = (lp * (d->n_pro - pp) + (d->n_lig - lp) * pp) / (double)K;
            I.w = 10 * kCostPair + (int)std::llround(10.0 * kCostDesolv * f);
        }
        I.u_begin = u;
        u += (I.k_end - I.k_begin) * (long long)I.w;
        k = I.k_end;
        tiles += nt;
        const size_t sm = smem_fixed(r.variant, r.P, G, r.block) +
                          (size_t)d->n_rows * d->n_types * record_bytes(r.variant, G, r.P) +
                          protein_bytes(r.variant, r.P, G) * (size_t)ch +
                          run_bytes(r.variant, r.P, G, d->n_types, d->n_lig);
        smem_max = std::max(smem_max, sm);
        pl->inst.push_back(I);
    }
    pl->n_total = k;
    pl->u_total = u;
    pl->n_tiles = tiles;
    pl->smem = smem_max;
    pl->fn = kernel_for(r.variant, r.P, G, r.cull != 0);
    if (pl->inst.empty()) return BUDE_OK;
    CK(raise_smem_limit(pl->fn, pl->smem), "shared-memory limit");
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pl->fn, r.block, pl->smem),
       "occupancy query");
    if (occ < 1) {
        cudaFuncAttributes fa;
        int regs = cudaFuncGetAttributes(&fa, pl->fn) == cudaSuccess ? fa.numRegs : -1;
        return fail(BUDE_ERR_UNSUPPORTED,
                    "block %d cannot be resident: %d registers per thread, %zu B shared memory",
                    r.block, regs, pl->smem);
    }
    occ = std::min(occ, r.cps);
    long long grid = (long long)di.sms * occ;
    if (grid > pl->n_total) grid = pl->n_total;
    pl->grid = (int)split_grid(pl->inst, pl->u_total, grid);
    return BUDE_OK;
}

size_t partial_bytes_for(const Plan& pl, const Resolved& r, bool G)
{
    const size_t NV = G ? 7 : 1;
    return ((size_t)pl.grid + (size_t)pl.n_tiles) * NV * 32u * (size_t)r.P * sizeof(double);
}

int ensure_workspace(double** partial, size_t* pbytes, unsigned** counter, size_t* ccount,
                     size_t need_bytes, size_t need_count, cudaStream_t s)
{
    if (need_bytes > *pbytes) {
        if (*partial) {
            CK(cudaStreamSynchronize(s), "workspace sync");
            cudaFree(*partial);
            *partial = nullptr;
            *pbytes = 0;
        }
        size_t b = std::max(need_bytes, (size_t)1 << 16);
        CK(dev_alloc((void**)partial, b), "workspace allocation");
        *pbytes = b;
    }
    if (need_count > *ccount) {
        if (*counter) {
            CK(cudaStreamSynchronize(s), "workspace sync");
            cudaFree(*counter);
            *counter = nullptr;
            *ccount = 0;
        }
        size_t c = std::max(need_count, (size_t)1024);
        CK(dev_alloc((void**)counter, c * sizeof(unsigned)), "workspace allocation");
        CK(cudaMemsetAsync(*counter, 0, c * sizeof(unsigned), s), "workspace clear");
        *ccount = c;
    }
    return BUDE_OK;
}

// Device error word of BUDE_DEVICE_CHECKS builds: one per device, looked up
// once (its host-side symbol is only a stand-in for the device address).
#ifdef BUDE_DEVICE_CHECKS
static __device__ unsigned g_device_err;
#endif

unsigned* device_err_word()
{
#ifdef BUDE_DEVICE_CHECKS
    static std::mutex m;
    static std::map<int, unsigned*> ptrs;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(m);
    auto it = ptrs.find(dev);
    if (it != ptrs.end()) return it->second;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_err) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<unsigned*>(p);
    return static_cast<unsigned*>(p);
#else
    return nullptr;
#endif
}

// BUDE_DEVICE_CHECKS builds: wait for the call's kernels, read and clear the
// device error word.  Release builds: nothing.
int device_checks(cudaStream_t s)
{
#ifdef BUDE_DEVICE_CHECKS
    unsigned* w = device_err_word();
    if (!w) return fail(BUDE_ERR_CUDA, "device error word unavailable");
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, w, sizeof h, cudaMemcpyDeviceToHost, s), "error word read");
    CK(cudaStreamSynchronize(s), "error word sync");
    if (h) {
        CK(cudaMemsetAsync(w, 0, sizeof h, s), "error word clear");
        CK(cudaStreamSynchronize(s), "error word sync");
        return fail(BUDE_ERR_DEVICE_FLAG, "device check failed: bits %#x", h);
    }
#else
    (void)s;
#endif
    return BUDE_OK;
}

int launch_plan(const Plan& pl, const Resolved& r, const Instance* dev_table, double* partial,
                unsigned* counter, cudaStream_t s)
{
    Args a;
    memset(&a, 0, sizeof a);
    a.n_inst = (int)pl.inst.size();
    if (a.n_inst == 1) a.single = pl.inst[0];
    a.table = dev_table;
    a.n_total = pl.n_total;
    // one deck: the units all cost the same, split by count
    a.u_total = a.n_inst > 1 ? pl.u_total : 0;
    a.partial = partial;
    a.counter = counter;
    a.err = device_err_word();
    a.n_slots = (long long)pl.grid + pl.n_tiles;
    a.n_tiles = pl.n_tiles;
    a.smem_bytes = pl.smem;
    void* params[] = {&a};
    CK(cudaLaunchKernel(pl.fn, dim3(pl.grid), dim3(r.block), params, pl.smem, s), "kernel launch");
    ++g_launches;
    return BUDE_OK;
}

int current_device(int* dev)
{
    CK(cudaGetDevice(dev), "cudaGetDevice");
    return BUDE_OK;
}

// Single-deck energies or adjoint.
int run_single(bude_deck* deck, const float* poses, int64_t n, float* energies, float* grad,
               const bude_options* opts, void* stream, bool G)
{
    g_launches = 0;
    if (!deck) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n < 0) return fail(BUDE_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return BUDE_OK;
    if (!poses) return fail(BUDE_ERR_INVALID_ARG, "poses is NULL");
    if (!G && !energies) return fail(BUDE_ERR_INVALID_ARG, "energies is NULL");
    if (G && !grad) return fail(BUDE_ERR_INVALID_ARG, "grad is NULL");
    Resolved r;
    int rc = resolve_options(opts, G, &r);
    if (rc) return rc;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    if (dev != deck->device)
        return fail(BUDE_ERR_INVALID_ARG, "deck lives on device %d, current device is %d",
                    deck->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const long long K = (long long)deck->n_lig * deck->n_pro;
    if (K == 0) {
        if (energies) CK(cudaMemsetAsync(energies, 0, (size_t)n * sizeof(float), s), "memset");
        if (G) CK(cudaMemsetAsync(grad, 0, (size_t)n * 6 * sizeof(float), s), "memset");
        return BUDE_OK;
    }
    Plan pl;
    rc = make_plan({deck}, {poses}, {(long long)n}, {energies}, {grad}, r, G, dev, &pl);
    if (rc) return rc;
    rc = ensure_workspace(&deck->partial, &deck->partial_bytes, &deck->counter,
                          &deck->counter_count, partial_bytes_for(pl, r, G), (size_t)pl.n_tiles,
                          s);
    if (rc) return rc;
    rc = launch_plan(pl, r, nullptr, deck->partial, deck->counter, s);
    if (rc) return rc;
    return device_checks(s);
}

// ---- caches of captured plans ----------------------------------------------
//
// Batched and refinement calls capture a CUDA graph per argument set and
// replay it.  A cache keeps at most kMaxCachedPlans of them and drops the
// least recently used when a new one comes in.  Callers hold a shared_ptr
// while they enqueue a replay, so a plan that another thread drops is
// destroyed only after that; a plan's destructor waits for the device before
// it frees the buffers a replay still in flight may use.  The caches are
// never destroyed (no CUDA calls at process exit).

constexpr size_t kMaxCachedPlans = 64;

template <typename K, typename P>
struct PlanCache {
    std::mutex m;
    std::map<K, std::pair<std::shared_ptr<P>, unsigned long long>> map;
    unsigned long long clock = 0;

    std::shared_ptr<P> find(const K& k)
    {
        std::lock_guard<std::mutex> lk(m);
        auto it = map.find(k);
        if (it == map.end()) return nullptr;
        it->second.second = ++clock;
        return it->second.first;
    }
    // Adds p unless another thread added a plan for k first; returns the
    // cached plan.  The plan dropped to make room is released after the lock.
    std::shared_ptr<P> insert(const K& k, std::shared_ptr<P> p)
    {
        std::shared_ptr<P> dropped;
        std::lock_guard<std::mutex> lk(m);
        auto ins = map.emplace(k, std::make_pair(p, ++clock));
        if (!ins.second) {
            ins.first->second.second = clock;
            return ins.first->second.first;
        }
        if (map.size() > kMaxCachedPlans) {
            auto oldest = map.begin();
            for (auto it = map.begin(); it != map.end(); ++it)
                if (it->second.second < oldest->second.second) oldest = it;
            dropped = std::move(oldest->second.first);
            map.erase(oldest);
        }
        return p;
    }
    // Drops every plan for which f(plan) holds (outside the lock).
    template <typename F>
    void drop_if(F f)
    {
        std::vector<std::shared_ptr<P>> dropped;
        {
            std::lock_guard<std::mutex> lk(m);
            for (auto it = map.begin(); it != map.end();) {
                if (f(*it->second.first)) {
                    dropped.push_back(std::move(it->second.first));
                    it = map.erase(it);
                } else {
                    ++it;
                }
            }
        }
    }
    size_t size()
    {
        std::lock_guard<std::mutex> lk(m);
        return map.size();
    }
};

// ---- batched plans -------------------------------------------------------

struct BatchKey {
    int dev;
    Resolved r;
    std::vector<const void*> ptrs;  // deck, poses, out per instance
    std::vector<long long> n;
    bool operator<(const BatchKey& o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (memcmp(&r, &o.r, sizeof r)) return memcmp(&r, &o.r, sizeof r) < 0;
        if (ptrs != o.ptrs) return ptrs < o.ptrs;
        return n < o.n;
    }
};

struct BatchPlan {
    Plan pl;
    Resolved r;
    std::vector<const bude_deck*> decks;
    Instance* dev_table = nullptr;
    double* partial = nullptr;
    size_t partial_bytes = 0;
    unsigned* counter = nullptr;
    size_t counter_count = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    ~BatchPlan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dev_table || partial || counter) cudaDeviceSynchronize();   // replays in flight
        if (dev_table) cudaFree(dev_table);
        if (partial) cudaFree(partial);
        if (counter) cudaFree(counter);
    }
};

PlanCache<BatchKey, BatchPlan>& g_batches = *new PlanCache<BatchKey, BatchPlan>;

void drop_batches_using(const bude_deck* d)
{
    g_batches.drop_if([d](const BatchPlan& bp) {
        return std::find(bp.decks.begin(), bp.decks.end(), d) != bp.decks.end();
    });
}

}  // namespace

static void drop_refines_using(const bude_deck* d);

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* bude_status_string(int status)
{
    switch (status) {
    case BUDE_OK: return "ok";
    case BUDE_ERR_INVALID_ARG: return "invalid argument";
    case BUDE_ERR_CUDA: return "CUDA error";
    case BUDE_ERR_OOM: return "out of device memory";
    case BUDE_ERR_UNSUPPORTED: return "unsupported shape or option";
    case BUDE_ERR_DEVICE_FLAG: return "device-side check failed";
    }
    return "unknown status";
}

const char* bude_last_error(void) { return g_last_error.c_str(); }

int bude_debug_fail_alloc(int32_t n)
{
    if (n < 0) return fail(BUDE_ERR_INVALID_ARG, "bude_debug_fail_alloc: n = %d < 0", n);
    g_fail_alloc_in.store(n);
    return BUDE_OK;
}

int32_t bude_debug_pending_fail_alloc(void) { return g_fail_alloc_in.load(); }

int64_t bude_last_launch_count(void) { return g_launches; }

int bude_get_default_options(int32_t variant, bude_options* out)
{
    if (!out || variant < 0 || variant > 3) return fail(BUDE_ERR_INVALID_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(g_opt_mutex);
    *out = g_default[variant];
    return BUDE_OK;
}

int bude_set_default_options(const bude_options* o)
{
    if (!o || o->variant < 0 || o->variant > 3) return fail(BUDE_ERR_INVALID_ARG, "bad options");
    Resolved r;
    int rc = resolve_options(o, false, &r);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_opt_mutex);
    g_default[o->variant] = {r.variant, r.P, r.block, r.tile, r.cps, r.cull};
    return BUDE_OK;
}

int bude_create_deck(const bude_deck_desc* desc, void* stream, bude_deck** out)
{
    Range range_("bude_create_deck");
    g_launches = 0;
    if (!out) return fail(BUDE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(BUDE_ERR_INVALID_ARG, "desc is NULL");
    if (desc->n_lig < 0 || desc->n_pro < 0)
        return fail(BUDE_ERR_INVALID_ARG, "negative atom count");
    if (desc->n_types < 1 || desc->n_types > BUDE_MAX_TYPES)
        return fail(BUDE_ERR_INVALID_ARG, "n_types %d outside 1..%d", desc->n_types,
                    BUDE_MAX_TYPES);
    if ((desc->n_lig && !desc->lig_xyzt) || (desc->n_pro && !desc->pro_xyzt) || !desc->ff)
        return fail(BUDE_ERR_INVALID_ARG, "NULL array with non-zero size");
    cudaStream_t s = (cudaStream_t)stream;
    bude_deck* d = new bude_deck;
    int rc = current_device(&d->device);
    if (rc) { delete d; return rc; }
    d->n_lig = desc->n_lig;
    d->n_pro = desc->n_pro;
    d->n_types = desc->n_types;
    struct Tmp { unsigned err; int n_rows; int lig_polar; int pro_polar; float centre[4]; };
    Tmp* tmp = nullptr;
    auto cleanup = [&](int code) {
        if (tmp) cudaFree(tmp);
        bude_destroy_deck(d);
        return code;
    };
#define CKD(call, what)                                               \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, what));   \
    } while (0)
    const size_t nl = std::max(1, d->n_lig), np = std::max(1, d->n_pro);
    const size_t pairs = (size_t)std::max(1, d->n_lig < d->n_types ? d->n_lig : d->n_types) *
                         d->n_types;
    CKD(dev_alloc((void**)&d->pro, np * sizeof(float4)), "deck allocation");
    CKD(dev_alloc((void**)&d->pro_c, np * sizeof(float4)), "deck allocation");
    CKD(dev_alloc((void**)&d->lig, nl * sizeof(float4)), "deck allocation");
    CKD(dev_alloc((void**)&d->tabF, pairs * sizeof(PairF)), "deck allocation");
    CKD(dev_alloc((void**)&d->tabG, pairs * sizeof(PairG)), "deck allocation");
    CKD(dev_alloc((void**)&d->tabD, pairs * sizeof(PairD)), "deck allocation");
    CKD(dev_alloc((void**)&d->row_type, (size_t)d->n_types * sizeof(int)), "deck allocation");
    CKD(dev_alloc((void**)&d->ff, (size_t)d->n_types * sizeof(float4)), "deck allocation");
    CKD(cudaMemcpyAsync(d->ff, desc->ff, (size_t)d->n_types * sizeof(float4),
                        cudaMemcpyDeviceToDevice, s), "forcefield copy");
    CKD(dev_alloc((void**)&tmp, sizeof(Tmp)), "deck allocation");
    CKD(cudaMemsetAsync(tmp, 0, sizeof(Tmp), s), "memset");
    CKD(launch_pack_protein((const float4*)desc->pro_xyzt, d->pro, d->n_pro, d->n_types,
                            &tmp->err, s),
        "protein packing launch");
    CKD(launch_build_tables((const float4*)desc->lig_xyzt, d->n_lig, (const float4*)desc->ff,
                            d->n_types, d->lig, d->tabF, d->tabG, d->tabD, d->row_type,
                            &tmp->n_rows, &tmp->err, s),
        "pair table launch");
    CKD(launch_count_polar((const float4*)desc->lig_xyzt, d->n_lig, d->ff, d->n_types,
                           &tmp->lig_polar, s),
        "polar count launch");
    CKD(launch_count_polar(d->pro, d->n_pro, d->ff, d->n_types, &tmp->pro_polar, s),
        "polar count launch");
    CKD(launch_recentre_protein(d->pro, d->pro_c, d->n_pro, tmp->centre, s),
        "protein recentring launch");
    g_launches += ((d->n_pro > 0) ? 3 : 1) + (d->n_lig > 0) + (d->n_pro > 0);
    Tmp h{0, 0, 0, 0, {0.f, 0.f, 0.f, 0.f}};
    CKD(cudaMemcpyAsync(&h, tmp, sizeof h, cudaMemcpyDeviceToHost, s), "readback");
    CKD(cudaStreamSynchronize(s), "deck synchronisation");
#undef CKD
    cudaFree(tmp);
    tmp = nullptr;
    if (h.err) {
        std::string why;
        if (h.err & 1u) why += " atom type outside [0, n_types);";
        if (h.err & 2u) why += " non-finite atom coordinate;";
        if (h.err & 4u) why += " forcefield row with radius <= 0, a non-finite value or hbtype not in {0,1,2};";
        bude_destroy_deck(d);
        return fail(BUDE_ERR_INVALID_ARG, "deck rejected:%s", why.c_str());
    }
    d->n_rows = h.n_rows;
    d->lig_polar = h.lig_polar;
    d->pro_polar = h.pro_polar;
    for (int j = 0; j < 3; ++j) d->centre[j] = h.centre[j];
    *out = d;
    return BUDE_OK;
}

int bude_destroy_deck(bude_deck* d)
{
    Range range_("bude_destroy_deck");
    if (!d) return BUDE_OK;
    drop_batches_using(d);
    drop_refines_using(d);
    cudaDeviceSynchronize();
    cudaFree(d->pro);
    cudaFree(d->pro_c);
    cudaFree(d->lig);
    cudaFree(d->tabF);
    cudaFree(d->tabG);
    cudaFree(d->tabD);
    cudaFree(d->row_type);
    cudaFree(d->ff);
    cudaFree(d->partial);
    cudaFree(d->counter);
    cudaFree(d->io);
    delete d;
    return BUDE_OK;
}

int bude_deck_info(const bude_deck* d, int32_t* n_lig, int32_t* n_pro, int32_t* n_types,
                   int32_t* n_rows)
{
    if (!d) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n_lig) *n_lig = d->n_lig;
    if (n_pro) *n_pro = d->n_pro;
    if (n_types) *n_types = d->n_types;
    if (n_rows) *n_rows = d->n_rows;
    return BUDE_OK;
}

int bude_energies(bude_deck* deck, const float* poses, int64_t n, float* energies,
                  const bude_options* opts, void* stream)
{
    Range range_("bude_energies");
    return run_single(deck, poses, n, energies, nullptr, opts, stream, false);
}

int bude_energies_host(bude_deck* deck, const float* poses, int64_t n, float* energies,
                       const bude_options* opts, void* stream)
{
    Range range_("bude_energies_host");
    g_launches = 0;
    if (!deck) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n < 0) return fail(BUDE_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return BUDE_OK;
    if (!poses || !energies) return fail(BUDE_ERR_INVALID_ARG, "poses or energies is NULL");
    int rc, dev;
    if ((rc = current_device(&dev))) return rc;
    if (dev != deck->device)
        return fail(BUDE_ERR_INVALID_ARG, "deck lives on device %d, current device is %d",
                    deck->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = (size_t)n * 7;
    if (need > deck->io_floats) {
        if (deck->io) {
            CK(cudaStreamSynchronize(s), "staging sync");
            cudaFree(deck->io);
            deck->io = nullptr;
            deck->io_floats = 0;
        }
        CK(dev_alloc((void**)&deck->io, need * sizeof(float)), "staging allocation");
        deck->io_floats = need;
    }
    float* dp = deck->io;
    float* de = deck->io + (size_t)n * 6;
    CK(cudaMemcpyAsync(dp, poses, (size_t)n * 6 * sizeof(float), cudaMemcpyHostToDevice, s),
       "pose upload");
    rc = run_single(deck, dp, n, de, nullptr, opts, stream, false);
    if (rc) return rc;
    const int64_t launches = g_launches;
    CK(cudaMemcpyAsync(energies, de, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s),
       "energy download");
    g_launches = launches;
    return BUDE_OK;
}

int bude_pose_grad(bude_deck* deck, const float* poses, int64_t n, float* energies, float* grad,
                   const bude_options* opts, void* stream)
{
    Range range_("bude_pose_grad");
    return run_single(deck, poses, n, energies, grad, opts, stream, true);
}

int bude_energies_batched(bude_deck* const* decks, const float* const* poses, const int64_t* n,
                          float* const* energies, int32_t count, const bude_options* opts,
                          void* stream)
{
    Range range_("bude_energies_batched");
    g_launches = 0;
    if (count < 0) return fail(BUDE_ERR_INVALID_ARG, "count %d < 0", count);
    if (count == 0) return BUDE_OK;
    if (!decks || !poses || !n || !energies)
        return fail(BUDE_ERR_INVALID_ARG, "NULL argument array");
    Resolved r;
    int rc = resolve_options(opts, false, &r);
    if (rc) return rc;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    BatchKey key;
    key.dev = dev;
    key.r = r;
    for (int i = 0; i < count; ++i) {
        if (!decks[i]) return fail(BUDE_ERR_INVALID_ARG, "decks[%d] is NULL", i);
        if (n[i] < 0) return fail(BUDE_ERR_INVALID_ARG, "n[%d] < 0", i);
        if (n[i] > 0 && (!poses[i] || !energies[i]))
            return fail(BUDE_ERR_INVALID_ARG, "NULL poses or energies for instance %d", i);
        if (decks[i]->device != dev)
            return fail(BUDE_ERR_INVALID_ARG, "decks[%d] lives on another device", i);
        key.ptrs.push_back(decks[i]);
        key.ptrs.push_back(poses[i]);
        key.ptrs.push_back(energies[i]);
        key.n.push_back(n[i]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::shared_ptr<BatchPlan> bp = g_batches.find(key);
    if (!bp) {
        bp = std::make_shared<BatchPlan>();
        bp->r = r;
        std::vector<const bude_deck*> dv(decks, decks + count);
        std::vector<const float*> pv(poses, poses + count);
        std::vector<long long> nv(n, n + count);
        std::vector<float*> ov(energies, energies + count);
        std::vector<float*> gv(count, nullptr);
        bp->decks = dv;
        rc = make_plan(dv, pv, nv, ov, gv, r, false, dev, &bp->pl);
        if (rc) return rc;
        const Plan& pl = bp->pl;
        auto bail = [](int code) { return code; };   // bp frees what it holds
        if (!pl.inst.empty()) {
            cudaError_t e = dev_alloc((void**)&bp->dev_table, pl.inst.size() * sizeof(Instance));
            if (e) return bail(cuda_fail(e, "plan allocation"));
            e = cudaMemcpy(bp->dev_table, pl.inst.data(), pl.inst.size() * sizeof(Instance),
                           cudaMemcpyHostToDevice);
            if (e) return bail(cuda_fail(e, "plan upload"));
            rc = ensure_workspace(&bp->partial, &bp->partial_bytes, &bp->counter,
                                  &bp->counter_count, partial_bytes_for(pl, r, false),
                                  (size_t)pl.n_tiles, s);
            if (rc) return bail(rc);
            e = cudaStreamSynchronize(s);
            if (e) return bail(cuda_fail(e, "plan synchronisation"));
        }
        // capture: zero-fill of instances without work, then the persistent launch
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e) return bail(cuda_fail(e, "capture stream"));
        device_err_word();  // resolve the check word's address before capturing
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e) { cudaStreamDestroy(cs); return bail(cuda_fail(e, "begin capture")); }
        int launches = 0;
        for (int i = 0; i < count; ++i) {
            const long long K = (long long)decks[i]->n_lig * decks[i]->n_pro;
            if (n[i] > 0 && K == 0) {
                cudaMemsetAsync(energies[i], 0, (size_t)n[i] * sizeof(float), cs);
            }
        }
        int lrc = BUDE_OK;
        if (!pl.inst.empty()) {
            int64_t saved = g_launches;
            lrc = launch_plan(pl, r, bp->dev_table, bp->partial, bp->counter, cs);
            launches = (int)(g_launches - saved);
        }
        e = cudaStreamEndCapture(cs, &bp->graph);
        cudaStreamDestroy(cs);
        if (lrc) return bail(lrc);
        if (e) return bail(cuda_fail(e, "end capture"));
        e = cudaGraphInstantiate(&bp->exec, bp->graph, 0);
        if (e) return bail(cuda_fail(e, "graph instantiation"));
        bp->launches = launches;
        // a plan another thread finished first for the same key wins; ours goes
        bp = g_batches.insert(key, bp);
    }
    CK(cudaGraphLaunch(bp->exec, s), "graph launch");
    g_launches = bp->launches;
    return device_checks(s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free energies: the same persistent kernel as bude_energies, with
// its cross-CTA partial sums and arrival tickets in a fixed device array
// that lives as long as the library is loaded.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticPartialDoubles = 512u * 1024u;  // 4 MiB of partial sums
constexpr size_t kStaticTickets = 16u * 1024u;          // 64 KiB of arrival tickets

struct StaticScratch {
    double partial[kStaticPartialDoubles];
    unsigned counter[kStaticTickets];
};

// Held by every GPU that loads libbude.so, from load until process exit.
static __device__ __align__(256) StaticScratch g_static_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
StaticScratch* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
int static_scratch(int dev, StaticScratch** out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return fail(BUDE_ERR_UNSUPPORTED, "device ordinal %d above %d", dev, kMaxDevices - 1);
    std::lock_guard<std::mutex> lk(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress");
        g_static_ptr[dev] = static_cast<StaticScratch*>(p);
    }
    *out = g_static_ptr[dev];
    return BUDE_OK;
}

}  // namespace

extern "C" BUDE_API int bude_energies_noalloc(bude_deck* deck, const float* poses, int64_t n,
                                              float* energies, const bude_options* opts,
                                              void* stream)
{
    Range range_("bude_energies_noalloc");
    g_launches = 0;
    if (!deck) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n < 0) return fail(BUDE_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return BUDE_OK;
    if (!poses || !energies) return fail(BUDE_ERR_INVALID_ARG, "poses or energies is NULL");
    Resolved r;
    int rc = resolve_options(opts, false, &r);
    if (rc) return rc;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    if (dev != deck->device)
        return fail(BUDE_ERR_INVALID_ARG, "deck lives on device %d, current device is %d",
                    deck->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    if ((long long)deck->n_lig * deck->n_pro == 0) {
        CK(cudaMemsetAsync(energies, 0, (size_t)n * sizeof(float), s), "memset");
        return BUDE_OK;
    }
    Plan pl;
    rc = make_plan({deck}, {poses}, {(long long)n}, {energies}, {nullptr}, r, false, dev, &pl);
    if (rc) return rc;
    const size_t need_doubles = partial_bytes_for(pl, r, false) / sizeof(double);
    if (need_doubles > kStaticPartialDoubles || (size_t)pl.n_tiles > kStaticTickets)
        return fail(BUDE_ERR_UNSUPPORTED,
                    "bude_energies_noalloc: %lld poses need %zu partial sums and %lld tickets; "
                    "its fixed scratch holds %zu and %zu (use fewer poses per call, or "
                    "bude_energies)",
                    (long long)n, need_doubles, pl.n_tiles, kStaticPartialDoubles,
                    kStaticTickets);
    StaticScratch* sc = nullptr;
    if ((rc = static_scratch(dev, &sc))) return rc;
    // tickets must start at zero; the partial sums are written before read
    CK(cudaMemsetAsync(sc->counter, 0, (size_t)pl.n_tiles * sizeof(unsigned), s),
       "ticket clear");
    rc = launch_plan(pl, r, nullptr, sc->partial, sc->counter, s);
    if (rc) return rc;
    return device_checks(s);
}

// ---------------------------------------------------------------------------
// On-device pose refinement: steps of adjoint + propose + accept, captured
// once into a CUDA graph per argument set and replayed.
// ---------------------------------------------------------------------------
namespace {

constexpr float kRefineGrow = 1.25f;
constexpr float kRefineShrink = 0.5f;

struct RefineKey {
    int dev;
    Resolved r;
    const void* deck;
    const void* poses;
    const void* energies;
    long long n;
    int steps;
    float step0;
    bool operator<(const RefineKey& o) const { return memcmp(this, &o, sizeof *this) < 0; }
};

// The plan owns every buffer its graph uses, the partial-sum workspace
// included: the deck's own workspace is reallocated when a later call on the
// deck needs more, and a captured graph would keep the freed address.
struct RefinePlan {
    float* buf = nullptr;  // E[n] g[6n] trial[6n] Et[n] gt[6n] alpha[n]
    double* partial = nullptr;
    size_t partial_bytes = 0;
    unsigned* counter = nullptr;
    size_t counter_count = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const bude_deck* deck = nullptr;
    int launches = 0;
    ~RefinePlan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (buf || partial || counter) cudaDeviceSynchronize();   // replays in flight
        if (buf) cudaFree(buf);
        if (partial) cudaFree(partial);
        if (counter) cudaFree(counter);
    }
};

PlanCache<RefineKey, RefinePlan>& g_refines = *new PlanCache<RefineKey, RefinePlan>;

}  // namespace

static void drop_refines_using(const bude_deck* d)
{
    g_refines.drop_if([d](const RefinePlan& rp) { return rp.deck == d; });
}

extern "C" BUDE_API int bude_debug_cached_plans(int32_t* batched, int32_t* refine)
{
    if (batched) *batched = (int32_t)g_batches.size();
    if (refine) *refine = (int32_t)g_refines.size();
    return BUDE_OK;
}

extern "C" BUDE_API int bude_refine(bude_deck* deck, float* poses, int64_t n, int32_t steps,
                                    float step0, float* energies, const bude_options* opts,
                                    void* stream)
{
    Range range_("bude_refine");
    g_launches = 0;
    if (!deck) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n < 0 || steps < 0) return fail(BUDE_ERR_INVALID_ARG, "negative n or steps");
    if (!(step0 > 0.f) || !std::isfinite(step0))
        return fail(BUDE_ERR_INVALID_ARG, "step0 must be positive and finite");
    if (n == 0) return BUDE_OK;
    if (!poses || !energies) return fail(BUDE_ERR_INVALID_ARG, "poses or energies is NULL");
    Resolved r;
    int rc = resolve_options(opts, true, &r);
    if (rc) return rc;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    if (dev != deck->device)
        return fail(BUDE_ERR_INVALID_ARG, "deck lives on device %d, current device is %d",
                    deck->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    if ((long long)deck->n_lig * deck->n_pro == 0) {
        CK(cudaMemsetAsync(energies, 0, (size_t)n * sizeof(float), s), "memset");
        return BUDE_OK;
    }
    RefineKey key;
    memset(&key, 0, sizeof key);
    key.dev = dev;
    key.r = r;
    key.deck = deck;
    key.poses = poses;
    key.energies = energies;
    key.n = n;
    key.steps = steps;
    key.step0 = step0;
    std::shared_ptr<RefinePlan> rp = g_refines.find(key);
    if (!rp) {
        rp = std::make_shared<RefinePlan>();
        rp->deck = deck;
        auto bail = [](int code) { return code; };   // rp frees what it holds
        const size_t N = (size_t)n;
        cudaError_t e = dev_alloc((void**)&rp->buf, 22 * N * sizeof(float));
        if (e) return bail(cuda_fail(e, "refine buffers"));
        float* E = rp->buf;
        float* g = E + N;
        float* trial = g + 6 * N;
        float* Et = trial + 6 * N;
        float* gt = Et + N;
        float* alpha = gt + 6 * N;
        Plan p0, p1;
        rc = make_plan({deck}, {poses}, {(long long)n}, {E}, {g}, r, true, dev, &p0);
        if (rc) return bail(rc);
        rc = make_plan({deck}, {trial}, {(long long)n}, {Et}, {gt}, r, true, dev, &p1);
        if (rc) return bail(rc);
        rc = ensure_workspace(&rp->partial, &rp->partial_bytes, &rp->counter, &rp->counter_count,
                              std::max(partial_bytes_for(p0, r, true),
                                       partial_bytes_for(p1, r, true)),
                              (size_t)std::max(p0.n_tiles, p1.n_tiles), s);
        if (rc) return bail(rc);
        e = cudaStreamSynchronize(s);
        if (e) return bail(cuda_fail(e, "refine synchronisation"));
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e) return bail(cuda_fail(e, "capture stream"));
        device_err_word();  // resolve the check word's address before capturing
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e) { cudaStreamDestroy(cs); return bail(cuda_fail(e, "begin capture")); }
        int64_t saved = g_launches;
        int lrc = BUDE_OK;
        cudaError_t ke = launch_refine_init(alpha, n, step0, cs);
        ++g_launches;
        if (ke == cudaSuccess) lrc = launch_plan(p0, r, nullptr, rp->partial, rp->counter, cs);
        for (int it = 0; it < steps && ke == cudaSuccess && lrc == BUDE_OK; ++it) {
            ke = launch_refine_propose(poses, g, alpha, trial, n, cs);
            ++g_launches;
            if (ke != cudaSuccess) break;
            lrc = launch_plan(p1, r, nullptr, rp->partial, rp->counter, cs);
            if (lrc != BUDE_OK) break;
            ke = launch_refine_accept(poses, E, g, trial, Et, gt, alpha, n, kRefineGrow,
                                      kRefineShrink, cs);
            ++g_launches;
        }
        cudaError_t ce = cudaSuccess;
        if (ke == cudaSuccess && lrc == BUDE_OK)
            ce = cudaMemcpyAsync(energies, E, N * sizeof(float), cudaMemcpyDeviceToDevice, cs);
        rp->launches = (int)(g_launches - saved);
        e = cudaStreamEndCapture(cs, &rp->graph);
        cudaStreamDestroy(cs);
        if (lrc) return bail(lrc);
        if (ke) return bail(cuda_fail(ke, "refine kernel launch"));
        if (ce) return bail(cuda_fail(ce, "refine energy copy"));
        if (e) return bail(cuda_fail(e, "end capture"));
        e = cudaGraphInstantiate(&rp->exec, rp->graph, 0);
        if (e) return bail(cuda_fail(e, "graph instantiation"));
        rp = g_refines.insert(key, rp);
    }
    CK(cudaGraphLaunch(rp->exec, s), "graph launch");
    g_launches = rp->launches;
    return device_checks(s);
}

// ---------------------------------------------------------------------------
// Gradient of sum_k w_k E_k with respect to ligand coordinates and forcefield
// ---------------------------------------------------------------------------
extern "C" BUDE_API int bude_param_grad(bude_deck* deck, const float* poses, int64_t n,
                                        const float* weights, float* lig_grad, float* ff_grad,
                                        const bude_options* opts, void* stream)
{
    Range range_("bude_param_grad");
    g_launches = 0;
    if (!deck) return fail(BUDE_ERR_INVALID_ARG, "deck is NULL");
    if (n < 0) return fail(BUDE_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (!lig_grad && deck->n_lig > 0) return fail(BUDE_ERR_INVALID_ARG, "lig_grad is NULL");
    if (!ff_grad) return fail(BUDE_ERR_INVALID_ARG, "ff_grad is NULL");
    if (n > 0 && !poses) return fail(BUDE_ERR_INVALID_ARG, "poses is NULL");
    Resolved r;
    int rc = resolve_options(opts, true, &r);
    if (rc) return rc;
    if (r.variant == BUDE_FP64)
        return fail(BUDE_ERR_UNSUPPORTED, "bude_param_grad has FP32 variants only");
    const int kv = r.variant == BUDE_FP32_FAST ? kFAST : kIEEE;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    if (dev != deck->device)
        return fail(BUDE_ERR_INVALID_ARG, "deck lives on device %d, current device is %d",
                    deck->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const long long K = (long long)deck->n_lig * deck->n_pro;
    if (n == 0 || K == 0) {
        if (deck->n_lig) CK(cudaMemsetAsync(lig_grad, 0, (size_t)deck->n_lig * 3 * sizeof(float), s), "memset");
        CK(cudaMemsetAsync(ff_grad, 0, (size_t)deck->n_types * 3 * sizeof(float), s), "memset");
        return BUDE_OK;
    }
    const void* fn = kernel_param(kv, r.P);
    if (!fn) return fail(BUDE_ERR_UNSUPPORTED, "poses per thread %d not built for bude_param_grad", r.P);
    const DeviceInfo di = device_info(dev);
    const size_t budget = smem_budget(di, r.cps);
    const size_t fixed = param_smem_bytes(r.P, deck->n_lig, deck->n_rows, deck->n_types, 0);
    const size_t atom_bytes = (size_t)param_atom_bytes(r.P);
    if (fixed + atom_bytes * 32 > budget)
        return fail(BUDE_ERR_UNSUPPORTED, "gradient accumulators and pair table do not fit in shared memory");
    int chunk = (int)std::min<size_t>((size_t)deck->n_pro, (budget - fixed) / atom_bytes);
    if (r.tile > 0) chunk = std::min(chunk, r.tile);
    const size_t smem = param_smem_bytes(r.P, deck->n_lig, deck->n_rows, deck->n_types, chunk);
    CK(raise_smem_limit(fn, smem), "shared-memory limit");
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, r.block, smem), "occupancy query");
    if (occ < 1) return fail(BUDE_ERR_UNSUPPORTED, "block %d cannot be resident", r.block);
    const long long TP = 32ll * r.P;
    const long long tiles = (n + TP - 1) / TP;
    const long long N = tiles * K;
    long long grid = (long long)di.sms * std::min(occ, r.cps);
    if (grid > N) grid = N;
    const int acc_len = deck->n_lig * 3 + deck->n_rows * deck->n_types * 3;
    const size_t need = ((size_t)grid + 1) * (size_t)acc_len * sizeof(double);
    rc = ensure_workspace(&deck->partial, &deck->partial_bytes, &deck->counter,
                          &deck->counter_count, need, 0, s);
    if (rc) return rc;
    ParamArgs a;
    memset(&a, 0, sizeof a);
    a.pro = deck->pro_c;
    a.ox = deck->centre[0];
    a.oy = deck->centre[1];
    a.oz = deck->centre[2];
    a.lig = deck->lig;
    a.pair = deck->tabG;
    a.poses = poses;
    a.weights = weights;
    a.n_poses = n;
    a.n_total = N;
    a.cta_acc = deck->partial;
    a.n_lig = deck->n_lig;
    a.n_pro = deck->n_pro;
    a.n_types = deck->n_types;
    a.n_rows = deck->n_rows;
    a.chunk = chunk;
    void* params[] = {&a};
    CK(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(r.block), params, smem, s), "kernel launch");
    double* sums = deck->partial + (size_t)grid * acc_len;
    CK(launch_param_reduce(deck->partial, (int)grid, deck->n_lig, deck->n_rows, deck->n_types,
                           sums, deck->row_type, deck->ff, lig_grad, ff_grad, s),
       "reduction launch");
    g_launches = 3;
    return device_checks(s);
}

// ---------------------------------------------------------------------------
// Test hook: the persistent kernel's work split, computed on the host by the
// functions the kernel and the planner use (no CUDA call).
// ---------------------------------------------------------------------------
extern "C" BUDE_API int bude_debug_partition(int32_t count, const int64_t* K, const int64_t* nt,
                                             const int32_t* w, int32_t grid, int32_t* grid_out,
                                             int64_t* cta_begin, int64_t* owner, int32_t* cover)
{
    if (count < 1 || !K || !nt || !w || grid < 1 || !grid_out)
        return fail(BUDE_ERR_INVALID_ARG, "bude_debug_partition: bad arguments");
    std::vector<Instance> inst;
    long long k = 0, u = 0, tiles = 0;
    for (int i = 0; i < count; ++i) {
        if (K[i] < 1 || nt[i] < 1 || w[i] < 1)
            return fail(BUDE_ERR_INVALID_ARG, "bude_debug_partition: instance %d is empty", i);
        Instance I;
        memset(&I, 0, sizeof I);
        I.k_begin = k;
        I.k_end = k + nt[i] * K[i];
        I.tile_begin = tiles;
        I.w = w[i];
        I.u_begin = u;
        u += (I.k_end - I.k_begin) * (long long)I.w;
        k = I.k_end;
        tiles += nt[i];
        inst.push_back(I);
    }
    const long long C = split_grid(inst, u, std::min<long long>(grid, k));
    *grid_out = (int32_t)C;
    // the launch parameters the kernel would see (launch_plan)
    Args a;
    memset(&a, 0, sizeof a);
    a.n_inst = count;
    a.single = inst[0];
    a.table = inst.data();
    a.n_total = k;
    a.u_total = count > 1 ? u : 0;
    const bool weighted = a.u_total > 0 && a.n_inst > 1;
    const long long N = a.n_total, U = a.u_total;
    // the same range and owner expressions as pose_kernel
    if (cta_begin) {
        for (long long c = 0; c < C; ++c)
            cta_begin[c] = weighted ? k_of_cost(a, (c * U + C - 1) / C) : c * N / C;
        cta_begin[C] = weighted ? k_of_cost(a, (C * U + C - 1) / C) : N;
    }
    for (size_t i = 0; i < inst.size(); ++i) {
        const Instance& I = inst[i];
        auto own = [&](long long kk) {
            return weighted ? owner_cta_weighted(kk, I, U, C) : owner_cta(kk, N, C);
        };
        if (owner)
            for (long long kk = I.k_begin; kk < I.k_end; ++kk) owner[kk] = own(kk);
        if (cover)
            for (long long t = 0; t < nt[i]; ++t) {
                const long long k0 = I.k_begin + t * K[i];
                cover[I.tile_begin + t] = (int32_t)(own(k0 + K[i] - 1) - own(k0) + 1);
            }
    }
    return BUDE_OK;
}
