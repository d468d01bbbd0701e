// goc_api.cu -- host side of the C ABI declared in include/goc.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/goc.h"
#include "goc_aux.cuh"
#include "goc_device.cuh"
#include "goc_std.cuh"
#include "goc_step.cuh"
#include "goc_internal.h"

using namespace goc;

// Named ranges for timeline tools (NVTX; no cost without an attached tool).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

namespace {

thread_local std::string g_err;

goc_status fail(goc_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

size_t elem_size(int storage) { return storage == GOC_FP32 ? 4 : 2; }

constexpr int kGraphSteps = 64;  // steps per captured graph (even: one buffer cycle per 2)
constexpr int kRefEvery = 1024;  // default steps between refreshes of the per-row storage reference
constexpr int kSlabGhost = 2;     // ghost rows per internal cut of a slab

}  // namespace

goc_status goc_fail(goc_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fail(st, "%s", buf);
}


namespace {

// ---- TMA descriptors -------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        cudaGetLastError();
    }
    return fn;
}

// 3D map [planes][ny][nx] of a population buffer (row pitch `pitch` elements),
// box [planes][by][bx]; out-of-range elements read as zero.
bool encode_planes(CUtensorMap *m, int storage, void *base, int nx, int ny, int pitch, int planes, int bx, int by) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || !base) return false;
    const cuuint64_t es = storage == GOC_FP32 ? 4 : 2;
    const CUtensorMapDataType dt = storage == GOC_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : storage == GOC_FP16_DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * ny * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class S>
bool encode_lattice_maps(goc_lattice *L) {
    using T = Tiling<S>;
    bool ok = true;
    for (int b = 0; b < 2; b++) {
        ok = ok && encode_planes(&L->tmf[b], L->storage, L->f[b], L->nx, L->ny, L->pitch, 9, T::BX, T::BY);
        ok = ok && encode_planes(&L->tmF[b], L->storage, L->F[b], L->nx, L->ny, L->pitch, 2, T::BX, T::BY);
        ok = ok && encode_planes(&L->tmf2[b], L->storage, L->f[b], L->nx, L->ny, L->pitch, 9, T::BX, Tiling2<S>::BY);
        ok = ok && encode_planes(&L->tmF2[b], L->storage, L->F[b], L->nx, L->ny, L->pitch, 2, T::BX, Tiling2<S>::BY);
        if (L->mhd.enabled)
            ok = ok && encode_planes(&L->tmg[b], L->storage, L->g[b], L->nx, L->ny, L->pitch, 10, T::BX, T::BYG);
    }
    return ok;
}


StepParams params_for(goc_lattice *L, int src, float *uout) {
    StepParams p = L->sp;
    p.fin = L->f[src];
    p.fout = L->f[src ^ 1];
    p.Fin = L->F[src];
    p.Fout = L->F[src ^ 1];
    p.gin = L->g[src];
    p.gout = L->g[src ^ 1];
    p.uout = uout;
    p.sr = (L->storage != GOC_FP32 && L->rounding == 0) ? 1 : 0;
    p.seed_rd = reinterpret_cast<const unsigned *>(L->flag + 2 + src);
    p.seed_wr = reinterpret_cast<unsigned *>(L->flag + 2 + (src ^ 1));
    static const bool static_tiles = std::getenv("GOC_STATIC_TILES") != nullptr;
    p.tctr = (static_tiles || !L->cfg_dynamic) ? nullptr : L->flag + 4 + src;
    p.tctr_next = L->flag + 4 + (src ^ 1);
    p.use_tma = L->tma_ok ? 1 : 0;
    if (L->tma_ok) {
        p.tm_f = L->tmf[src];
        p.tm_F = L->tmF[src];
        if (L->mhd.enabled) p.tm_g = L->tmg[src];
    }
    return p;
}

// Zero the tile queues of both parities after steps of a batch kernel, which
// leaves them as they were (called outside graph capture).
goc_status clean_queues(goc_lattice *L) {
    if (!L->queues_dirty) return GOC_OK;
    CU(cudaMemsetAsync(L->flag + 4, 0, 2 * sizeof(int), L->stream));
    L->queues_dirty = false;
    return GOC_OK;
}

goc_status launch_one(goc_lattice *L, float *uout) {
    if (goc_status st = clean_queues(L); st != GOC_OK) return st;
    StepParams p = params_for(L, L->cur, uout);
    p.nopull = L->fresh ? 1 : 0;
    goc_status st;
    if (L->aa) {
        switch (L->storage) {
            case GOC_FP16_DEV: st = launch_aa_step_t<__half>(L, p); break;
            case GOC_BF16_DEV: st = launch_aa_step_t<__nv_bfloat16>(L, p); break;
            default: st = launch_aa_step_t<float>(L, p); break;
        }
    } else {
        switch (L->storage) {
            case GOC_FP16_DEV: st = launch_step_t<__half>(L, p); break;
            case GOC_BF16_DEV: st = launch_step_t<__nv_bfloat16>(L, p); break;
            default: st = launch_step_t<float>(L, p); break;
        }
    }
    if (st != GOC_OK) return st;
    L->cur ^= 1;
    L->steps++;
    L->fresh = false;
    return GOC_OK;
}

// ---- launch autotuner ------------------------------------------------------
// Candidates: tile queue or static order x the balanced grid x dependent
// launch on or off -- on straight grids with the central-moment collision the
// tile height (8 or 16 rows) in place of the last, with dependent launch on;
// the standard scheme has no tiles (dependent launch only).  Each runs 2 + 16 real steps of the lattice; the 16 are timed
// with CUDA events.  Every candidate gives bitwise the same populations.
constexpr long long kTuneWarm = 2, kTuneSteps = 16;
std::mutex g_tune_mu;
std::map<std::array<int, 5>, std::array<int, 4>> g_tune_cache;

bool tile_rows_apply(const goc_lattice *L) { return L->scheme == 0 && L->sp.curv == 0; }

goc_status autotune(goc_lattice *L, long long *nsteps) {
    if (L->tuned) return GOC_OK;
    const std::array<int, 5> key = {L->nx, L->ny, L->storage, L->mhd.enabled ? 1 : 0, L->scheme};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            L->cfg_dynamic = it->second[0];
            L->cfg_pdl = it->second[1];
            L->cfg_balanced = it->second[2];
            L->cfg_rows = it->second[3];
            L->tuned = true;
            return GOC_OK;
        }
    }
    // (straight grids with the central-moment collision: the tile height takes
    // the place of the dependent-launch switch, which measured best on everywhere)
    const bool rows = tile_rows_apply(L);
    const int ncand = L->scheme == 1 ? 2 : 8;
    if (*nsteps < ncand * (kTuneWarm + kTuneSteps)) return GOC_OK;   // tune on a longer call
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bd = 1, bp = 1, bb = 0, br = 1;
    goc_status st = GOC_OK;
    for (int c = 0; c < ncand && st == GOC_OK; c++) {
        L->cfg_pdl = (c & 1) && !rows ? 0 : 1;
        L->cfg_rows = (c & 1) && rows ? 2 : 1;
        L->cfg_dynamic = (c & 2) ? 0 : 1;
        L->cfg_balanced = (c & 4) ? 1 : 0;
        for (long long s = 0; s < kTuneWarm && st == GOC_OK; s++) st = launch_one(L, nullptr);
        cudaEventRecord(e0, L->stream);
        for (long long s = 0; s < kTuneSteps && st == GOC_OK; s++) st = launch_one(L, nullptr);
        cudaEventRecord(e1, L->stream);
        if (st != GOC_OK) break;
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = fail(GOC_ECUDA, "autotuner timing failed");
            break;
        }
        *nsteps -= kTuneWarm + kTuneSteps;
        if (ms < best) {
            best = ms;
            bd = L->cfg_dynamic;
            bp = L->cfg_pdl;
            bb = L->cfg_balanced;
            br = L->cfg_rows;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GOC_OK) return st;
    L->cfg_dynamic = bd;
    L->cfg_pdl = bp;
    L->cfg_balanced = bb;
    L->cfg_rows = br;
    L->tuned = true;
    if (L->graph) {   // captured under another configuration
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {bd, bp, bb, br};
    return GOC_OK;
}

goc_status ensure_graph(goc_lattice *L) {
    if (goc_status st = clean_queues(L); st != GOC_OK) return st;
    if (L->graph) return GOC_OK;
    // capture kGraphSteps launches on a private stream (the lattice stream may
    // be the legacy default stream, which cannot be captured)
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = L->stream;
    int cur = L->cur;
    long long steps = L->steps;
    bool fresh = L->fresh;
    L->fresh = false;
    L->stream = cs;
    cudaGraph_t gr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    goc_status st = GOC_OK;
    if (e == cudaSuccess) {
        for (int k = 0; k < kGraphSteps && st == GOC_OK; k++) st = launch_one(L, nullptr);
        e = cudaStreamEndCapture(cs, &gr);
    }
    L->stream = keep;
    L->cur = cur;
    L->steps = steps;
    L->fresh = fresh;
    cudaStreamDestroy(cs);
    if (st != GOC_OK) return st;
    if (e != cudaSuccess) return fail(GOC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    L->graph_cur = cur;
    e = cudaGraphInstantiate(&L->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        L->graph = nullptr;
        return fail(GOC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    return GOC_OK;
}

goc_status validate(const goc_grid *grid, const goc_map *map) {
    if (!grid || !map) return fail(GOC_EINVAL, "grid and map are required");
    if (grid->nx < 1 || grid->ny < 1) return fail(GOC_EINVAL, "nx, ny must be >= 1 (got %d, %d)", grid->nx, grid->ny);
    if ((long long)grid->nx * grid->ny > (1LL << 31) || grid->ny > 65535)
        return fail(GOC_EINVAL, "lattice too large (nx*ny <= 2^31, ny <= 65535)");
    for (int s = 0; s < 4; s++)
        if (grid->bc[s] != GOC_BC_PERIODIC && grid->bc[s] != GOC_BC_WALL)
            return fail(GOC_EINVAL, "bc[%d] must be GOC_BC_PERIODIC or GOC_BC_WALL", s);
    for (int s = 0; s < 4; s++)
        if (!std::isfinite(grid->wall_u[s]) || !std::isfinite(grid->wall_b[s][0]) || !std::isfinite(grid->wall_b[s][1]))
            return fail(GOC_EINVAL, "wall speeds and fields must be finite");
    for (int a = 0; a < 2; a++) {
        const double mv[] = {map->beta[a], map->a[a], map->gamma[a], map->alpha[a], map->mu[a], map->yc[a]};
        for (double v : mv)
            if (!std::isfinite(v)) return fail(GOC_EINVAL, "map parameters must be finite");
    }
    if (!std::isfinite(map->r_inner) || !std::isfinite(map->r_outer) || !std::isfinite(map->sectors))
        return fail(GOC_EINVAL, "map parameters must be finite");
    if (grid->bc[0] != grid->bc[1] || grid->bc[2] != grid->bc[3])
        return fail(GOC_EINVAL, "opposite sides must both be periodic or both walls");
    if (grid->bc[0] == GOC_BC_WALL && grid->nx < 3) return fail(GOC_EINVAL, "a wall axis needs >= 3 nodes");
    if (grid->bc[2] == GOC_BC_WALL && grid->ny < 3) return fail(GOC_EINVAL, "a wall axis needs >= 3 nodes");
    if (map->kind[0] == GOC_MAP_TABLE) {   // general orthogonal grid given node by node
        if (!map->table || !map->wall_table) return fail(GOC_EINVAL, "the TABLE map needs table and wall_table");
        const long long N = (long long)grid->nx * grid->ny;
        for (long long n = 0; n < 2 * N; n++)
            if (!(map->table[n] > 0.0 && std::isfinite(map->table[n])))
                return fail(GOC_EINVAL, "TABLE: h1, h2 must be finite and > 0 at every node");
        for (long long n = 2 * N; n < 6 * N; n++)
            if (!std::isfinite(map->table[n])) return fail(GOC_EINVAL, "TABLE: theta must be finite");
        const int nw = 2 * grid->ny + 2 * grid->nx;
        for (int s = 0; s < 4; s++) {   // wall-normal and tangential metric of the wall sides
            if (grid->bc[s] != GOC_BC_WALL) continue;
            const int off = s < 2 ? s * grid->ny : 2 * grid->ny + (s - 2) * grid->nx, n = s < 2 ? grid->ny : grid->nx;
            for (int t = 0; t < 2; t++)
                for (int k = 0; k < n; k++) {
                    const double v = map->wall_table[t * nw + off + k];
                    if (!(v > 0.0 && std::isfinite(v)))
                        return fail(GOC_EINVAL, "TABLE: wall_table must be finite and > 0 along the walls");
                }
        }
        return GOC_OK;
    }
    for (int a = 0; a < 2; a++) {
        int k = map->kind[a];
        if (k == GOC_MAP_TABLE) return fail(GOC_EINVAL, "the TABLE map is given as kind[0]");
        if (k < 0 || k > 7) return fail(GOC_EINVAL, "map kind[%d] = %d unknown", a, k);
        int per = grid->bc[a == 0 ? 0 : 2] == GOC_BC_PERIODIC;
        if (k == GOC_MAP_ANNULUS) {
            if (a != 0) return fail(GOC_EINVAL, "the annulus map is a xi1 (radial) map");
            if (per || grid->bc[2] != GOC_BC_PERIODIC || map->kind[1] != GOC_MAP_UNIFORM)
                return fail(GOC_EINVAL, "the annulus needs W/E walls, periodic S/N and a uniform xi2 map");
            if (!(map->r_inner > 0.0 && map->r_outer > map->r_inner && map->sectors > 0.0))
                return fail(GOC_EINVAL, "the annulus needs 0 < r_inner < r_outer and sectors > 0");
            continue;
        }
        const bool wall_map = k == GOC_MAP_ROBERTS || k == GOC_MAP_TANH1 || k == GOC_MAP_SINH ||
                              (k == GOC_MAP_TANH2 && map->beta[a] != 0.0);
        if (wall_map && per) return fail(GOC_EINVAL, "axis %d: wall-clustering map on a periodic axis", a);
        if (k == GOC_MAP_TANH1 && !(map->beta[a] > 0.0)) return fail(GOC_EINVAL, "one-wall tanh beta must be > 0");
        if (k == GOC_MAP_SINH && !(map->mu[a] > 0.0 && map->mu[a] <= 50.0))
            return fail(GOC_EINVAL, "interior-map mu must be in (0, 50]");
        if (k == GOC_MAP_SINH && !(map->yc[a] > 0.0 && map->yc[a] < 1.0))
            return fail(GOC_EINVAL, "interior-map yc must be in (0, 1)");
        if (k == GOC_MAP_SINE && !per) return fail(GOC_EINVAL, "axis %d: sine map needs a periodic axis", a);
        if (k == GOC_MAP_SINE && !(std::fabs(map->a[a]) < 1.0)) return fail(GOC_EINVAL, "sine amplitude must be < 1");
        if (k == GOC_MAP_TANH2 && !(map->beta[a] >= 0.0)) return fail(GOC_EINVAL, "beta must be >= 0");
        if (k == GOC_MAP_ROBERTS && !(map->gamma[a] > 1.0)) return fail(GOC_EINVAL, "Roberts gamma must be > 1");
        if (k == GOC_MAP_ROBERTS && !(map->alpha[a] == 0.0 || map->alpha[a] == 0.5))
            return fail(GOC_EINVAL, "Roberts alpha must be 0 or 1/2");
    }
    return GOC_OK;
}

MapParams map_params(const goc_grid *grid, const goc_map *map, int axis) {
    MapParams m;
    m.kind = map->kind[axis];
    m.n = axis == 0 ? grid->nx : grid->ny;
    m.periodic = grid->bc[axis == 0 ? 0 : 2] == GOC_BC_PERIODIC;
    m.beta = map->beta[axis];
    m.a = map->a[axis];
    m.gamma = map->gamma[axis];
    m.alpha = map->alpha[axis];
    m.mu = map->mu[axis];
    m.yc = map->yc[axis];
    m.r_in = map->r_inner;
    m.r_out = map->r_outer;
    m.sectors = map->sectors;
    m.n2 = grid->ny;
    return m;
}

// Rows of a global xi2 axis metric g = [2][ng + 2] (h, theta at the nodes,
// then the walls at xi = 0 and ng) for a slab: local row k is global row
// first + k (wrapped on a periodic axis); the wall entries are the global
// walls where the slab reaches them, else the slab's edge rows (an internal
// cut, which only ghost rows see).
__global__ void slice_axis_kernel(const double *g, int ng, int first, int periodic, int wall_lo, int wall_hi,
                                  double *out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n + 2) return;
    int src;
    if (k < n) src = periodic ? ((first + k) % ng + ng) % ng : first + k;
    else if (k == n) src = wall_lo ? ng : first;
    else src = wall_hi ? ng + 1 : first + n - 1;
    out[k] = g[src];
    out[n + 2 + k] = g[ng + 2 + src];
}

// Two rows [row, row + 2) of every plane of the current buffers (populations,
// stored force, MIE populations) to or from a message buf[plane][2][nx].
template <class S>
__global__ void halo_kernel(const StepParams p, S *buf, int row, int unpack) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y, k = blockIdx.z;
    if (i >= p.nx) return;
    S *base = k < 9 ? static_cast<S *>(const_cast<void *>(p.fin)) + k * p.plane
                    : (k < 11 ? static_cast<S *>(const_cast<void *>(p.Fin)) + (k - 9) * p.plane
                              : static_cast<S *>(const_cast<void *>(p.gin)) + (k - 11) * p.plane);
    S *cell = base + (long long)(row + r) * p.pitch + i;
    S *msg = buf + ((long long)k * 2 + r) * p.nx + i;
    if (unpack) *cell = *msg;
    else *msg = *cell;
}

// The FP64 per-row storage reference rows [3][ny] of rows [row, row + 2) to or
// from msg[3][2].
__global__ void halo_ref_kernel(double *ref, int ny, double *msg, int row, int unpack) {
    const int t = threadIdx.x;
    if (t >= 6) return;
    const int c = t / 2, r = t % 2;
    if (unpack) ref[c * ny + row + r] = msg[t];
    else msg[t] = ref[c * ny + row + r];
}

// FP64 metric of both axes on the device: d1, d2 = [2][n+2] (h, theta); q.
// Annulus: d1 = [4][n1+2] (h1, theta11, h2, theta21 over xi1) and q is the
// smallest of h1 and h2 over the nodes.
goc_status compute_metric(const goc_grid *grid, const goc_map *map, cudaStream_t st,
                          double *d1, double *d2, double *qdev) {
    MapParams a = map_params(grid, map, 0), b = map_params(grid, map, 1);
    metric_axis_kernel<<<(b.n + 2 + 127) / 128, 128, 0, st>>>(b, d2, d2 + b.n + 2);
    if (a.kind == GOC_MAP_ANNULUS) {
        annulus_metric_kernel<<<(a.n + 2 + 127) / 128, 128, 0, st>>>(a, d1);
        min_h_kernel<<<1, 256, 0, st>>>(d1, a.n, d1 + 2 * (a.n + 2), a.n, qdev);
    } else {
        metric_axis_kernel<<<(a.n + 2 + 127) / 128, 128, 0, st>>>(a, d1, d1 + a.n + 2);
        min_h_kernel<<<1, 256, 0, st>>>(d1, a.n, d2, b.n, qdev);
    }
    CU(cudaGetLastError());
    return GOC_OK;
}

// Guard bands (debug aid in place of a memory checker): with GOC_GUARD_BANDS
// set at creation, the padding columns [nx, pitch) of every plane of the
// population, force and MIE buffers and a tail after each buffer hold the
// byte 0xA5; no kernel writes there, so goc_check_guards counting other bytes
// finds stray writes.
constexpr size_t kGuardTail = 65536;
constexpr unsigned char kCanary = 0xA5;
size_t guard_tail(const goc_lattice *L) { return L->guard ? kGuardTail : 0; }

__global__ void guard_kernel(unsigned char *buf, long long rows, long long row_bytes, long long valid_bytes,
                             long long tail_bytes, int check, unsigned long long *bad) {
    const long long padw = row_bytes - valid_bytes, pad = rows * padw, total = pad + tail_bytes;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const long long a = k < pad ? (k / padw) * row_bytes + valid_bytes + k % padw : rows * row_bytes + (k - pad);
        if (check) {
            if (buf[a] != kCanary) atomicAdd(bad, 1ull);
        } else {
            buf[a] = kCanary;
        }
    }
}

// Fill (check = false) or count (check = true, into *bad) the guard bytes of
// both buffers of every population array of L.
goc_status guard_pass(goc_lattice *L, bool check, long long *bad) {
    const long long es = (long long)elem_size(L->storage), row = L->pitch * es, valid = L->nx * es;
    unsigned long long *d = nullptr;
    if (check) {
        CU(cudaMalloc(&d, sizeof(unsigned long long)));
        CU(cudaMemsetAsync(d, 0, sizeof(unsigned long long), L->stream));
    }
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        void *bufs[3] = {L->f[b], L->F[b], L->g[b]};
        const int planes[3] = {9, 2, 10};
        for (int k = 0; k < 3 && e == cudaSuccess; k++) {
            if (!bufs[k]) continue;
            guard_kernel<<<148, 256, 0, L->stream>>>(static_cast<unsigned char *>(bufs[k]), (long long)planes[k] * L->ny,
                                                    row, valid, (long long)kGuardTail, check ? 1 : 0, d);
            e = cudaGetLastError();
        }
    }
    unsigned long long h = 0;
    if (e == cudaSuccess && check) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return fail(GOC_ECUDA, "guard pass failed: %s", cudaGetErrorString(e));
    if (bad) *bad = (long long)h;
    return GOC_OK;
}

// Self-test of the bounded device-side wait: one thread waits on an mbarrier
// that nothing completes, gives up after `polls` polls and records status 2,
// as the step kernels' waits do; the context stays usable.
__global__ void wait_selftest_kernel(long long polls, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    for (long long k = 0; k < polls; k++)
        if (mbar_try_wait(&bar, 0)) {
            *status = 0;
            return;
        }
    *status = 2;
}

// The device status word flag[0]: 1 = NaN/Inf or non-positive density seen
// by a step, 2 = a staged tile copy did not complete within its bounded wait.
goc_status flag_status(const goc_lattice *L, int f) {
    if (f == 1) return fail(GOC_EDIVERGED, "lattice diverged (by step %lld)", L->steps);
    if (f == 2) return fail(GOC_ETIMEOUT, "a staged tile copy did not complete within its bounded wait");
    return fail(GOC_ECUDA, "unknown device status %d", f);
}

// Read flag[0] after the stream has drained (synchronous, 4 bytes).
goc_status device_status(goc_lattice *L) {
    int f = 0;
    CU(cudaMemcpy(&f, L->flag, sizeof(int), cudaMemcpyDeviceToHost));
    return f ? flag_status(L, f) : GOC_OK;
}

void free_lattice(goc_lattice *L) {
    if (!L) return;
    cudaStreamSynchronize(L->stream);
    if (L->graph) cudaGraphExecDestroy(L->graph);
    if (L->aa) {   // one buffer, named twice
        L->f[1] = nullptr;
        L->F[1] = nullptr;
        L->g[1] = nullptr;
    }
    void *ptrs[] = {L->f[0], L->f[1], L->F[0], L->F[1], L->g[0], L->g[1], L->tab1, L->tab2,
                    L->m1, L->m2, L->gm, L->uout[0], L->uout[1], L->flag, L->red, L->mom,
                    L->ref64, L->reft, L->aa_fld, L->aa_wsum};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (L->flag_ev) cudaEventDestroy(L->flag_ev);
    if (L->hflag) cudaFreeHost(L->hflag);
    if (L->owns_stream && L->stream) cudaStreamDestroy(L->stream);
    delete L;
}

template <class T>
goc_status dalloc(goc_lattice *L, T **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? GOC_ENOMEM : GOC_ECUDA, "cudaMalloc(%zu) failed: %s",
                    bytes, cudaGetErrorString(e));
    }
    L->device_bytes += bytes;
    return GOC_OK;
}

// ---- per-row storage reference (16-bit storage, straight grids) -------------
// FP32 tables from the FP64 rows src ([3][ny]).
goc_status ref_tables(goc_lattice *L, const double *src) {
    const StepParams &p = L->sp;
    ref_tables_kernel<<<(L->ny + 127) / 128, 128, 0, L->stream>>>(
        L->m2, L->m2 + L->ny + 2, L->ny, p.per_y, L->flow.rho0, L->csm2, src, L->reft, L->reft + L->ny,
        L->reft + 3 * L->ny);
    CU(cudaGetLastError());
    return GOC_OK;
}

// The reference of a new state: A1 = 0, Bref = the initial uniform field.
goc_status ref_reset(goc_lattice *L) {
    const int ny = L->ny;
    const double v[3] = {0.0, L->mhd.enabled ? L->mhd.b_init[0] : 0.0, L->mhd.enabled ? L->mhd.b_init[1] : 0.0};
    for (int k = 0; k < 3; k++) {
        fill_kernel<<<(ny + 255) / 256, 256, 0, L->stream>>>(L->ref64 + (long long)k * ny, ny, v[k]);
        CU(cudaGetLastError());
    }
    return ref_tables(L, L->ref64);
}

// Refresh: row means of U1 and B of the current state become the reference,
// the stored values are re-expressed against it, the tables rebuilt.
goc_status ref_refresh(goc_lattice *L) {
    StepParams p = params_for(L, L->cur, nullptr);
    p.nopull = L->fresh ? 1 : 0;
    double *next = L->ref64 + 3 * (long long)L->ny;
    const dim3 ag((L->nx + 127) / 128, L->ny);
    const unsigned salt = (unsigned)L->steps * 0x9E3779B1u + 0x632BE5ABu;
    const double *h1 = L->m1, *t1 = L->m1 + L->nx + 2, *h2 = L->m2, *t2 = L->m2 + L->ny + 2;
    const double rho0 = L->flow.rho0, csm2 = L->csm2;
    const int pre = L->fresh ? 1 : 0;
    const bool m = L->mhd.enabled;
    const int lay = L->aa && !L->fresh ? (L->cur ? AA_S : AA_T) : AA_C;   // where the populations sit
#define GOC_REF_LAUNCH(S, MHD)                                                                                 \
    do {                                                                                                       \
        ref_rows_kernel<S, MHD><<<L->ny, 256, 0, L->stream>>>(p, next, pre, lay);                               \
        ref_apply_kernel<S, MHD><<<ag, 128, 0, L->stream>>>(p, h1, t1, h2, t2, next, rho0, csm2, pre, salt, lay); \
    } while (0)
    if (L->storage == GOC_FP16_DEV) {
        if (m) GOC_REF_LAUNCH(__half, true);
        else GOC_REF_LAUNCH(__half, false);
    } else {
        if (m) GOC_REF_LAUNCH(__nv_bfloat16, true);
        else GOC_REF_LAUNCH(__nv_bfloat16, false);
    }
#undef GOC_REF_LAUNCH
    CU(cudaGetLastError());
    goc_status st = ref_tables(L, next);
    if (st != GOC_OK) return st;
    CU(cudaMemcpyAsync(L->ref64, next, 3 * (size_t)L->ny * sizeof(double), cudaMemcpyDeviceToDevice, L->stream));
    return GOC_OK;
}

// Refresh when due (the step count reached ref_next).
goc_status ref_maybe_refresh(goc_lattice *L) {
    if (L->ref_every <= 0 || L->steps < L->ref_next) return GOC_OK;
    goc_status st = ref_refresh(L);
    L->ref_next = (L->steps / L->ref_every + 1) * L->ref_every;
    return st;
}

goc_status run_init(goc_lattice *L, const double *rho, const double *u1, const double *u2,
                    const double *b1, const double *b2, bool persistent_staging = false) {
    const long long N = (long long)L->nx * L->ny;
    if (L->aa) L->cur = 0;   // in place: the parity names the layout, and the first step reads f^0
    // staging of the given FP64 fields on the device: the moments buffer
    // (kept for later calls) when asked, else a temporary allocation; a field
    // not given is its default constant and takes no memory (so a lattice
    // created with uniform fields needs no staging beyond its own buffers)
    const double *src[5] = {rho, u1, u2, b1, b2};
    const double dflt[5] = {L->flow.rho0, 0.0, 0.0, L->mhd.b_init[0], L->mhd.b_init[1]};
    int given = 0;
    for (int k = 0; k < 5; k++) given += src[k] ? 1 : 0;
    double *dev = nullptr;
    bool temporary = false;
    if (given && persistent_staging) {
        if (!L->mom) {
            CU(cudaMalloc(&L->mom, 5 * N * sizeof(double)));
            L->device_bytes += 5 * N * sizeof(double);
        }
        dev = L->mom;
    } else if (given) {
        CU(cudaMalloc(&dev, given * N * sizeof(double)));
        temporary = true;
    }
    double *fld[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int cmask = 0, slot = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 5 && e == cudaSuccess; k++) {
        if (src[k]) {
            fld[k] = dev + slot++ * N;
            e = cudaMemcpyAsync(fld[k], src[k], N * sizeof(double), cudaMemcpyHostToDevice, L->stream);
        } else {
            cmask |= 1 << k;
        }
    }
    if (e != cudaSuccess) {
        if (temporary) cudaFree(dev);
        return fail(GOC_ECUDA, "init copy failed: %s", cudaGetErrorString(e));
    }
    if (L->ref64) {   // the initial state is expressed against the creation reference
        goc_status st = ref_reset(L);
        if (st != GOC_OK) {
            if (temporary) cudaFree(dev);
            return st;
        }
    }
    InitParams q;
    q.sp = params_for(L, L->cur, nullptr);   // writes the current buffer
    q.sp.fout = L->f[L->cur];
    q.sp.Fout = L->F[L->cur];
    q.sp.gout = L->g[L->cur];
    q.h1d = L->m1;
    q.h2x = L->sp.curv == 1 ? L->m1 + 2 * (L->nx + 2) : nullptr;
    q.t21x = L->sp.curv == 1 ? L->m1 + 3 * (L->nx + 2) : nullptr;
    q.t1d = L->m1 + L->nx + 2;
    q.h2d = L->m2;
    q.t2d = L->m2 + L->ny + 2;
    q.cs2 = L->cs2;
    q.nu = L->nu;
    q.zeta = L->zeta;
    q.rho0 = L->flow.rho0;
    q.csm2 = L->csm2;
    q.eta = L->eta;
    q.gi = L->flow.gi_correction;
    q.mhd = L->mhd.enabled;
    q.rho = fld[0];
    q.u1 = fld[1];
    q.u2 = fld[2];
    q.b1 = fld[3];
    q.b2 = fld[4];
    for (int k = 0; k < 5; k++) q.cval[k] = dflt[k];
    q.cmask = cmask;
    dim3 grid((L->nx + 127) / 128, L->ny), block(128);
    switch (L->storage) {
        case GOC_FP16_DEV: init_kernel<__half><<<grid, block, 0, L->stream>>>(q); break;
        case GOC_BF16_DEV: init_kernel<__nv_bfloat16><<<grid, block, 0, L->stream>>>(q); break;
        default: init_kernel<float><<<grid, block, 0, L->stream>>>(q); break;
    }
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(L->stream);
    if (temporary) cudaFree(dev);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(GOC_ECUDA, "init kernel failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    L->steps = 0;
    L->res_u = L->res_b = 0.0;
    L->fresh = true;
    if (cudaMemsetAsync(L->flag + 2, 0, 2 * sizeof(int), L->stream) != cudaSuccess ||   // step counters
        cudaMemsetAsync(L->flag, 0, sizeof(int), L->stream) != cudaSuccess)             // status word
        return fail(GOC_ECUDA, "memset failed");
    if (L->hflag) *L->hflag = 0;
    if (L->ref_every > 0) {   // reference from the initial fields
        goc_status st = ref_refresh(L);
        if (st != GOC_OK) return st;
        L->ref_next = L->ref_every;
    }
    return GOC_OK;
}

__global__ void to_float_kernel(const double *in, float *out, long long n) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) out[k] = (float)in[k];
}

// Macroscopic fields of the current state into L->mom ([5][ny][nx] FP64).
goc_status moments_to_device(goc_lattice *L) {
    const long long N = (long long)L->nx * L->ny;
    if (!L->mom) {
        CU(cudaMalloc(&L->mom, 5 * N * sizeof(double)));
        L->device_bytes += 5 * N * sizeof(double);
    }
    StepParams p = params_for(L, L->cur, nullptr);
    p.nopull = L->fresh ? 1 : 0;
    if (L->aa) {
        switch (L->storage) {
            case GOC_FP16_DEV: return launch_aa_moments_t<__half>(L, p, L->mom);
            case GOC_BF16_DEV: return launch_aa_moments_t<__nv_bfloat16>(L, p, L->mom);
            default: return launch_aa_moments_t<float>(L, p, L->mom);
        }
    }
    dim3 grid((L->nx + 127) / 128, L->ny), block(128);
    const bool m = L->mhd.enabled;
    switch (L->storage) {
        case GOC_FP16_DEV:
            if (m) moments_kernel<__half, true><<<grid, block, 0, L->stream>>>(p, L->mom);
            else moments_kernel<__half, false><<<grid, block, 0, L->stream>>>(p, L->mom);
            break;
        case GOC_BF16_DEV:
            if (m) moments_kernel<__nv_bfloat16, true><<<grid, block, 0, L->stream>>>(p, L->mom);
            else moments_kernel<__nv_bfloat16, false><<<grid, block, 0, L->stream>>>(p, L->mom);
            break;
        default:
            if (m) moments_kernel<float, true><<<grid, block, 0, L->stream>>>(p, L->mom);
            else moments_kernel<float, false><<<grid, block, 0, L->stream>>>(p, L->mom);
    }
    CU(cudaGetLastError());
    return GOC_OK;
}

}  // namespace

extern "C" {

const char *goc_last_error(void) { return g_err.c_str(); }

goc_status goc_check_guards(goc_lattice *L, long long *bad) {
    if (!L || !bad) return fail(GOC_EINVAL, "lattice and bad are required");
    if (!L->guard) return fail(GOC_EINVAL, "guard bands are off (set GOC_GUARD_BANDS before goc_create)");
    return guard_pass(L, true, bad);
}

goc_status goc_selftest_bounded_wait(long long polls) {
    if (polls < 1 || polls > (1LL << 26)) return fail(GOC_EINVAL, "polls must be in [1, 2^26]");
    int *d = nullptr, h = -1;
    CU(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(GOC_ECUDA, "wait self-test failed: %s", cudaGetErrorString(e));
    if (h == 2) return fail(GOC_ETIMEOUT, "the bounded wait ran out after %lld polls", polls);
    return fail(GOC_ECUDA, "wait self-test: unexpected status %d", h);
}

// Node-table metric: q = the smallest h1, h2 over the nodes (host table).
double table_q(const goc_grid *grid, const goc_map *map) {
    const long long N = (long long)grid->nx * grid->ny;
    double q = map->table[0];
    for (long long n = 0; n < 2 * N; n++) q = std::min(q, map->table[n]);
    return q;
}

goc_status goc_metric_info(const goc_grid *grid, const goc_map *map, double *q, double *cs2) {
    goc_status st = validate(grid, map);
    if (st != GOC_OK) return st;
    if (map->kind[0] == GOC_MAP_TABLE) {
        const double qh = table_q(grid, map);
        if (q) *q = qh;
        if (cs2) *cs2 = qh * qh / 3.0;
        return GOC_OK;
    }
    double *d = nullptr;
    size_t n1 = grid->nx + 2, n2 = grid->ny + 2;
    CU(cudaMalloc(&d, (4 * n1 + 2 * n2 + 1) * sizeof(double)));
    st = compute_metric(grid, map, 0, d, d + 4 * n1, d + 4 * n1 + 2 * n2);
    double qh = 0;
    cudaError_t e = cudaMemcpy(&qh, d + 4 * n1 + 2 * n2, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (st != GOC_OK) return st;
    if (e != cudaSuccess) return fail(GOC_ECUDA, "metric copy failed: %s", cudaGetErrorString(e));
    if (q) *q = qh;
    if (cs2) *cs2 = qh * qh / 3.0;
    return GOC_OK;
}

// A slab of a global lattice: its global xi2 extent and the rows it covers.
struct SlabPlan {
    const goc_grid *global;
    int r0, r1, glo, ghi;
};

static goc_status create_impl(const goc_grid *grid, const goc_map *map, const goc_flow *flow, const goc_mhd *mhd,
                              const goc_exec *exec, const SlabPlan *slab, goc_lattice **out);

goc_status goc_create(const goc_grid *grid, const goc_map *map, const goc_flow *flow,
                      const goc_mhd *mhd, const goc_exec *exec, goc_lattice **out) {
    return create_impl(grid, map, flow, mhd, exec, nullptr, out);
}

static goc_status create_impl(const goc_grid *grid, const goc_map *map, const goc_flow *flow, const goc_mhd *mhd,
                              const goc_exec *exec, const SlabPlan *slab, goc_lattice **out) {
    TraceRange trace_("goc_create");
    if (!out) return fail(GOC_EINVAL, "out is NULL");
    *out = nullptr;
    // (a slab's whole lattice was validated by goc_create_slab; its own xi2
    // sides are walls whatever the global axis is)
    goc_status st = slab ? GOC_OK : validate(grid, map);
    if (st != GOC_OK) return st;
    if (!flow) return fail(GOC_EINVAL, "flow is required");
    {   // every real parameter finite (a NaN passes the range checks below unnoticed)
        const double fv[] = {flow->rho0, flow->tau, flow->nu, flow->tau_zeta, flow->omega_free, flow->fext[0],
                             flow->fext[1]};
        for (double v : fv)
            if (!std::isfinite(v)) return fail(GOC_EINVAL, "flow parameters must be finite");
        if (mhd && mhd->enabled) {
            const double mv[] = {mhd->tau_m, mhd->eta, mhd->mu_m, mhd->b_init[0], mhd->b_init[1]};
            for (double v : mv)
                if (!std::isfinite(v)) return fail(GOC_EINVAL, "MIE parameters must be finite");
        }
    }
    if (!(flow->rho0 > 0.0)) return fail(GOC_EINVAL, "rho0 must be > 0");
    if (flow->nu <= 0.0 && !(flow->tau > 0.5)) return fail(GOC_EINVAL, "need nu > 0 or tau > 1/2");
    if (exec && (exec->storage < 0 || exec->storage > 2)) return fail(GOC_EINVAL, "unknown storage %d", exec->storage);
    if (exec && (exec->scheme < 0 || exec->scheme > 3)) return fail(GOC_EINVAL, "unknown scheme %d", exec->scheme);
    if (exec && exec->scheme == 1) {
        const bool uni = map && (map->kind[0] == GOC_MAP_UNIFORM || (map->kind[0] == GOC_MAP_TANH2 && map->beta[0] == 0.0)) &&
                         (map->kind[1] == GOC_MAP_UNIFORM || (map->kind[1] == GOC_MAP_TANH2 && map->beta[1] == 0.0));
        if (!uni) return fail(GOC_EINVAL, "the standard uniform-grid scheme needs uniform maps on both axes");
        if (flow->gi_correction) return fail(GOC_EINVAL, "the standard uniform-grid scheme needs gi_correction = 0");
        if (mhd && mhd->enabled) return fail(GOC_EINVAL, "the standard uniform-grid scheme has no MIE");
    }
    if (exec && (exec->streaming < 0 || exec->streaming > 1))
        return fail(GOC_EINVAL, "unknown streaming %d", exec->streaming);
    if (exec && exec->streaming == 1) {
        const bool straight = map->kind[0] != GOC_MAP_ANNULUS && map->kind[0] != GOC_MAP_TABLE;
        if (exec->scheme != 0 || !straight)
            return fail(GOC_EUNSUPPORTED, "in-place streaming needs scheme 0 and a straight grid");
    }
    goc_lattice *L = new (std::nothrow) goc_lattice();
    if (!L) return fail(GOC_ENOMEM, "host allocation failed");
    L->grid = *grid;
    L->map = *map;
    L->flow = *flow;
    if (L->flow.tau_zeta == 0.0) L->flow.tau_zeta = 1.0;
    if (L->flow.omega_free == 0.0) L->flow.omega_free = 1.0;
    std::memset(&L->mhd, 0, sizeof L->mhd);
    if (mhd && mhd->enabled) {
        L->mhd = *mhd;
        if (L->mhd.mu_m == 0.0) L->mhd.mu_m = 1.0;
        if (L->mhd.eta <= 0.0 && !(L->mhd.tau_m > 0.5)) {
            delete L;
            return fail(GOC_EINVAL, "MIE needs eta > 0 or tau_m > 1/2");
        }
    }
    if (exec) {
        L->storage = exec->storage;
        L->stream = (cudaStream_t)exec->cuda_stream;
        L->check_every = exec->check_every > 0 ? exec->check_every : 100;
        L->rounding = exec->rounding;
        L->scheme = exec->scheme;
        L->tuned = exec->fixed_launch != 0;
        L->aa = exec->streaming == 1;
        if (L->aa) L->tuned = true;   // its two launches per step have no tile order to tune
        L->plateau_checks = std::max(0, exec->plateau_checks);
        if (exec->device >= 0) {
            cudaError_t e = cudaSetDevice(exec->device);
            if (e != cudaSuccess) {
                delete L;
                return fail(GOC_ECUDA, "cudaSetDevice(%d): %s", exec->device, cudaGetErrorString(e));
            }
        }
    }
    cudaGetDevice(&L->device);
    L->nx = grid->nx;
    L->ny = grid->ny;
    L->guard = std::getenv("GOC_GUARD_BANDS") != nullptr;
    L->pitch = (grid->nx + 31) / 32 * 32;
    L->plane = (long long)L->pitch * L->ny;
    const size_t es = elem_size(L->storage);
#define TRY(x)                 \
    do {                       \
        goc_status s_ = (x);   \
        if (s_ != GOC_OK) {    \
            free_lattice(L);   \
            return s_;         \
        }                      \
    } while (0)
    for (int b = 0; b < (L->aa ? 1 : 2); b++) {
        TRY(dalloc(L, &L->f[b], 9 * L->plane * es + guard_tail(L)));
        TRY(dalloc(L, &L->F[b], 2 * L->plane * es + guard_tail(L)));
        if (L->mhd.enabled) TRY(dalloc(L, &L->g[b], 10 * L->plane * es + guard_tail(L)));
    }
    if (L->aa) {   // in place: one population and force buffer, the fields of the current step
        L->f[1] = L->f[0];
        L->F[1] = L->F[0];
        L->g[1] = L->g[0];
        L->aa_wn = std::max(L->nx, L->ny);
        TRY(dalloc(L, &L->aa_fld, 3 * L->plane * sizeof(float)));
        TRY(dalloc(L, &L->aa_wsum, 4 * (size_t)L->aa_wn * sizeof(float)));
    }
    const bool curv = map->kind[0] == GOC_MAP_ANNULUS;
    TRY(dalloc(L, &L->tab1, 16 * (size_t)L->nx * sizeof(float)));   // 8 rows, then the per-index records
    TRY(dalloc(L, &L->tab2, 16 * (size_t)L->ny * sizeof(float)));
    TRY(dalloc(L, &L->m1, (curv ? 4 : 2) * (size_t)(L->nx + 2) * sizeof(double)));
    TRY(dalloc(L, &L->m2, 2 * (size_t)(L->ny + 2) * sizeof(double)));
    TRY(dalloc(L, &L->flag, 8 * sizeof(int)));   // [0] status, [1] spare, [2..3] step counters, [4..5] tile queues of the two parities
    {   // pinned host copy of the status word and the event that marks its arrival
        cudaError_t e = cudaMallocHost((void **)&L->hflag, sizeof(int));
        if (e == cudaSuccess) {
            *L->hflag = 0;
            e = cudaEventCreateWithFlags(&L->flag_ev, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            free_lattice(L);
            return fail(GOC_ECUDA, "status word setup failed: %s", cudaGetErrorString(e));
        }
    }
    TRY(dalloc(L, &L->red, 8 * sizeof(double)));
    // metric (FP64), q, cs2 (Eq. GOC-LBE_CFL); a node table fills the axis
    // tables with a uniform metric (unused by its step kernel)
    const bool table = map->kind[0] == GOC_MAP_TABLE;
    goc_map uni_map = *map;
    if (table) uni_map.kind[0] = uni_map.kind[1] = GOC_MAP_UNIFORM;
    if (slab) {   // the global xi2 metric and q, then this slab's rows of it
        const int ng = slab->global->ny;
        double *m2g = nullptr;
        if (cudaMalloc(&m2g, 2 * (size_t)(ng + 2) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            free_lattice(L);
            return fail(GOC_ENOMEM, "slab metric staging failed");
        }
        goc_status ms = compute_metric(slab->global, map, L->stream, L->m1, m2g, L->red);
        if (ms == GOC_OK) {
            slice_axis_kernel<<<(L->ny + 2 + 127) / 128, 128, 0, L->stream>>>(
                m2g, ng, slab->r0 - slab->glo, slab->global->bc[2] == GOC_BC_PERIODIC, slab->glo == 0,
                slab->ghi == 0, L->m2, L->ny);
            if (cudaGetLastError() != cudaSuccess) ms = fail(GOC_ECUDA, "slab metric kernel failed");
        }
        cudaStreamSynchronize(L->stream);
        cudaFree(m2g);
        TRY(ms);
        L->slab = true;
        L->slab_r0 = slab->r0;
        L->slab_r1 = slab->r1;
        L->slab_glo = slab->glo;
        L->slab_ghi = slab->ghi;
    } else {
        TRY(compute_metric(grid, table ? &uni_map : map, L->stream, L->m1, L->m2, L->red));
    }
    double hw1[2], hw2[2], qh, hwt1[2] = {1.0, 1.0};
    {
        cudaError_t e = cudaMemcpyAsync(&qh, L->red, sizeof(double), cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw1, L->m1 + L->nx, 2 * sizeof(double), cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw2, L->m2 + L->ny, 2 * sizeof(double), cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess && curv)   // annulus: h2 at the radial walls (tangential factor)
            e = cudaMemcpyAsync(hwt1, L->m1 + 2 * (L->nx + 2) + L->nx, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                L->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) {
            free_lattice(L);
            return fail(GOC_ECUDA, "metric readback failed: %s", cudaGetErrorString(e));
        }
    }
    if (table) qh = table_q(grid, map);
    L->q = qh;
    L->cs2 = qh * qh / 3.0;
    if (L->flow.nu > 0.0) {
        L->nu = L->flow.nu;
        L->tau = L->nu / L->cs2 + 0.5;
    } else {
        L->tau = L->flow.tau;
        L->nu = L->cs2 * (L->tau - 0.5);
    }
    L->zeta = L->scheme == 2 ? L->nu : L->cs2 * (L->flow.tau_zeta - 0.5);   // SRT: zeta = nu
    if (L->mhd.enabled) {
        L->csm2 = L->cs2;   // c_sm = c_s (Eq. GOC-LBE_CFL-MIE)
        if (L->mhd.eta > 0.0) {
            L->eta = L->mhd.eta;
            L->taum = L->eta / L->csm2 + 0.5;
        } else {
            L->taum = L->mhd.tau_m;
            L->eta = L->csm2 * (L->taum - 0.5);
        }
    }
    // wall-normal metric at each wall: W/E -> h1(0), h1(n); S/N -> h2(0), h2(n)
    L->hw[0] = hw1[0];
    L->hw[1] = hw1[1];
    L->hw[2] = hw2[0];
    L->hw[3] = hw2[1];
    const double rho0cs2 = L->flow.rho0 * L->cs2;
    const int per_x = grid->bc[0] == GOC_BC_PERIODIC, per_y = grid->bc[2] == GOC_BC_PERIODIC;
    if (curv)
        annulus_tables_kernel<<<(L->nx + 127) / 128, 128, 0, L->stream>>>(L->m1, L->nx, rho0cs2, L->tab1);
    else
        axis_tables_kernel<<<(L->nx + 127) / 128, 128, 0, L->stream>>>(L->m1, L->m1 + L->nx + 2, L->nx, per_x,
                                                                       rho0cs2, L->cs2, L->tab1);
    axis_tables_kernel<<<(L->ny + 127) / 128, 128, 0, L->stream>>>(L->m2, L->m2 + L->ny + 2, L->ny, per_y, rho0cs2,
                                                                   L->cs2, L->tab2);
    axis_records_kernel<<<(L->nx + 127) / 128, 128, 0, L->stream>>>(L->tab1, L->nx);
    axis_records_kernel<<<(L->ny + 127) / 128, 128, 0, L->stream>>>(L->tab2, L->ny);
    if (table) {   // node-table metric: FP32 planes + walls for the step (and the initial state), the
                   // link corrections formed in FP64 from a temporary device copy of the table
        const long long N = (long long)L->nx * L->ny;
        const int wmax = std::max(L->nx, L->ny);
        TRY(dalloc(L, &L->gm, (10 * L->plane + 8 * (long long)wmax) * sizeof(float)));
        double *gtab = nullptr;
        {
            cudaError_t e = cudaMalloc(&gtab, 6 * N * sizeof(double));
            if (e != cudaSuccess) {
                cudaGetLastError();
                free_lattice(L);
                return fail(e == cudaErrorMemoryAllocation ? GOC_ENOMEM : GOC_ECUDA, "node-table staging: %s",
                            cudaGetErrorString(e));
            }
        }
        std::vector<float> walls(8 * (size_t)wmax, 1.f);
        const int nw = 2 * L->ny + 2 * L->nx;
        for (int t = 0; t < 2; t++) {   // t = 0: wall-normal factor, 1: tangential
            const double *w = map->wall_table + t * nw;
            float *o = walls.data() + 4 * t * (size_t)wmax;
            for (int k = 0; k < L->ny; k++) {
                o[k] = (float)w[k];                       // W (over j)
                o[wmax + k] = (float)w[L->ny + k];        // E
            }
            for (int k = 0; k < L->nx; k++) {
                o[2 * wmax + k] = (float)w[2 * L->ny + k];            // S (over i)
                o[3 * wmax + k] = (float)w[2 * L->ny + L->nx + k];    // N
            }
        }
        cudaError_t e = cudaMemsetAsync(L->gm, 0, 10 * L->plane * sizeof(float), L->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(gtab, map->table, 6 * N * sizeof(double), cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(L->gm + 10 * L->plane, walls.data(), walls.size() * sizeof(float),
                                cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess) {
            table_metric_kernel<<<dim3((L->nx + 127) / 128, L->ny), 128, 0, L->stream>>>(
                gtab, L->nx, L->ny, L->pitch, L->plane, per_x, per_y, rho0cs2, L->gm);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);   // the host arrays may go after return
        if (e != cudaSuccess) cudaStreamSynchronize(L->stream);
        cudaFree(gtab);
        if (e != cudaSuccess) {
            free_lattice(L);
            return fail(GOC_ECUDA, "node-table upload failed: %s", cudaGetErrorString(e));
        }
    }
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            free_lattice(L);
            return fail(GOC_ECUDA, "table kernel failed: %s", cudaGetErrorString(e));
        }
    }
    // step parameters
    StepParams &p = L->sp;
    std::memset(&p, 0, sizeof p);
    p.nx = L->nx;
    p.ny = L->ny;
    p.pitch = L->pitch;
    p.plane = L->plane;
    p.per_x = per_x;
    p.per_y = per_y;
    auto axis = [](float *t, int n) {
        Axis a;
        a.h = t;
        a.ih = t + n;
        a.th = t + 2 * n;
        a.rm = t + 3 * n;
        a.rp = t + 4 * n;
        a.dm = t + 5 * n;
        a.dp = t + 6 * n;
        return a;
    };
    p.ax1 = axis(L->tab1, L->nx);
    p.ax2 = axis(L->tab2, L->ny);
    p.curv = table ? 2 : curv ? 1 : 0;   // 1: the xi1 table then holds h2, 1/h2, theta21 in rows 5-7
    p.gm = L->gm;
    p.rho0 = (float)L->flow.rho0;
    p.cs2 = (float)L->cs2;
    p.ics2 = (float)(1.0 / L->cs2);
    p.nu = (float)L->nu;
    p.zeta = (float)L->zeta;
    for (int k = 0; k < 9; k++) p.om[k] = (float)L->flow.omega_free;
    p.om[3] = (float)(1.0 / L->flow.tau_zeta);
    p.om[4] = p.om[5] = (float)(1.0 / L->tau);
    if (L->scheme == 2)   // SRT: one rate for every moment
        for (int k = 0; k < 9; k++) p.om[k] = (float)(1.0 / L->tau);
    p.fext1 = (float)L->flow.fext[0];
    p.fext2 = (float)L->flow.fext[1];
    p.seed_row0 = L->slab ? L->slab_r0 - L->slab_glo : 0;
    p.own0 = L->slab ? L->slab_glo : 0;
    p.own1 = L->slab ? L->ny - L->slab_ghi : L->ny;
    p.gi = L->flow.gi_correction ? 1.f : 0.f;
    p.constF = L->scheme == 1 ? 1 : 0;
    p.zc = (float)(L->zeta / L->cs2);
    p.nc = (float)(L->nu / L->cs2);
    p.zmn = (float)(L->zeta - L->nu);
    p.A3 = (float)(2.0 * L->zeta + L->nu);
    p.A4 = (float)(L->zeta + 2.0 * L->nu);
    p.gic = (float)((L->flow.gi_correction ? 1.0 : 0.0) / L->cs2);
    for (int s = 0; s < 4; s++) {
        p.uw[s] = grid->bc[s] == GOC_BC_WALL ? (float)grid->wall_u[s] : 0.f;
        p.hwn[s] = (float)L->hw[s];
        if (p.uw[s] != 0.f) p.moving = 1;
        // the column metric's MIE wall condition takes h1 h2 at the wall: its
        // tangential factor h2 (constant along the radial walls) is folded in here
        const double ht = (curv && s < 2) ? hwt1[s] : 1.0;
        p.bw[s][0] = (float)(ht * grid->wall_b[s][0]);
        p.bw[s][1] = (float)(ht * grid->wall_b[s][1]);
    }
    // storage scales (1 for FP32; for 16-bit a per-lattice velocity scale)
    p.sf = p.isf = p.sF = p.isF = p.sg = p.isg = 1.f;
    if (L->storage != GOC_FP32) {
        double uref = 1e-3 * std::sqrt(L->cs2);   // (a slab takes the whole lattice's walls: one scale for all slabs)
        for (int s = 0; s < 4; s++)
            uref = std::max(uref, std::fabs(slab ? (slab->global->bc[s] == GOC_BC_WALL ? (double)(float)slab->global->wall_u[s] : 0.0)
                                                 : (double)p.uw[s]));
        {   // a body force drives flows up to about the Poiseuille centreline speed F n^2 / (8 nu)
            // across the lattice's extent n (the whole lattice's for a slab)
            const goc_grid *gg = slab ? slab->global : grid;
            const double fx = std::max(std::fabs(L->flow.fext[0]), std::fabs(L->flow.fext[1]));
            const double n = (double)std::max(gg->nx, gg->ny);
            if (fx > 0.0 && L->nu > 0.0) uref = std::max(uref, fx * n * n / (8.0 * L->nu));
        }
        double hmax = 1.0;   // scale so that |deviation| / s stays well inside the 16-bit range
        double sf = L->flow.rho0 * uref * hmax / 256.0;
        p.sf = (float)sf;
        p.isf = (float)(1.0 / sf);
        p.sF = (float)sf;   // the stored force deviation starts at h rho0 cs2 theta (F = 0 before step 1)
        p.isF = (float)(1.0 / sf);
        p.sg = (float)sf;
        p.isg = (float)(1.0 / sf);
    }
    if (L->mhd.enabled) {
        p.csm2 = (float)L->csm2;
        p.icsm2 = (float)(1.0 / L->csm2);
        p.taum = (float)L->taum;
        p.itaum = (float)(1.0 / L->taum);
        p.eta = (float)L->eta;
        p.imum = (float)(1.0 / L->mhd.mu_m);
        p.W0 = (float)(1.0 - 2.0 * L->csm2);
        p.W1 = (float)(0.5 * L->csm2);
        // storage reference field: the initial uniform field on straight grids;
        // curvilinear grids store g itself (B_rest = 0)
        p.brest[0] = p.curv ? 0.f : (float)L->mhd.b_init[0];
        p.brest[1] = p.curv ? 0.f : (float)L->mhd.b_init[1];
        double bmax = std::max(std::fabs(L->mhd.b_init[0]), std::fabs(L->mhd.b_init[1]));
        if (p.curv)
            for (int s = 0; s < 4; s++)
                if (grid->bc[s] == GOC_BC_WALL)
                    bmax = std::max(bmax, std::max(std::fabs(grid->wall_b[s][0]), std::fabs(grid->wall_b[s][1])));
        if (L->storage != GOC_FP32 && bmax > 0) {
            p.sg = (float)(bmax / 256.0);
            p.isg = (float)(256.0 / bmax);
        }
    }
    p.flag = L->flag;
    if (L->storage != GOC_FP32 && p.curv == 0) {   // per-row storage reference of 16-bit straight grids
        TRY(dalloc(L, &L->ref64, 6 * (size_t)L->ny * sizeof(double)));
        TRY(dalloc(L, &L->reft, 7 * (size_t)L->ny * sizeof(float)));
        p.reft = L->reft;
        const int every = exec ? exec->reference_every : 0;
        L->ref_every = (L->scheme == 1 || every < 0) ? 0 : (every > 0 ? every : kRefEvery);
    }
    switch (L->storage) {
        case GOC_FP16_DEV: L->tma_ok = encode_lattice_maps<__half>(L); break;
        case GOC_BF16_DEV: L->tma_ok = encode_lattice_maps<__nv_bfloat16>(L); break;
        default: L->tma_ok = encode_lattice_maps<float>(L); break;
    }
    if (std::getenv("GOC_DISABLE_TMA")) L->tma_ok = false;
    TRY(run_init(L, nullptr, nullptr, nullptr, nullptr, nullptr));
    if (L->guard) TRY(guard_pass(L, false, nullptr));
    {
        cudaError_t e = cudaMemsetAsync(L->flag, 0, 8 * sizeof(int), L->stream);
        if (e != cudaSuccess) {
            free_lattice(L);
            return fail(GOC_ECUDA, "memset failed");
        }
    }
#undef TRY
    *out = L;
    return GOC_OK;
}

goc_status goc_init_fields(goc_lattice *L, const double *rho, const double *u1, const double *u2,
                           const double *b1, const double *b2) {
    TraceRange trace_("goc_init_fields");
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    return run_init(L, rho, u1, u2, b1, b2, true);
}

void goc_destroy(goc_lattice *L) { free_lattice(L); }

static goc_status enqueue_steps(goc_lattice *L, long long nsteps);

goc_status goc_step(goc_lattice *L, long long nsteps) {
    TraceRange trace_("goc_step");
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (nsteps < 0) return fail(GOC_EINVAL, "nsteps must be >= 0");
    if (L->in_batch) return fail(GOC_EINVAL, "this lattice belongs to a batch: step it with goc_batch_step");
    if (L->slab && nsteps > 1)
        return fail(GOC_EINVAL, "a slab exchanges its ghost rows after every step: goc_step(slab, 1), then "
                                "goc_slab_pack / goc_slab_unpack");
    // the status word as of the end of the previous call, if its copy has landed (no wait)
    if (L->flag_ev && cudaEventQuery(L->flag_ev) == cudaSuccess && *L->hflag) return flag_status(L, *L->hflag);
    goc_status st = enqueue_steps(L, nsteps);
    if (st != GOC_OK) return st;
    if (L->flag_ev) {   // refresh the host copy of the status word behind this call's work
        CU(cudaMemcpyAsync(L->hflag, L->flag, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
        CU(cudaEventRecord(L->flag_ev, L->stream));
    }
    return GOC_OK;
}

static goc_status enqueue_run(goc_lattice *L, long long nsteps);

// Steps in runs that end where a refresh of the per-row storage reference is
// due (every ref_every steps), so the refresh points depend only on the step
// count.
static goc_status enqueue_steps(goc_lattice *L, long long nsteps) {
    if (L->ref_every <= 0) return enqueue_run(L, nsteps);
    while (nsteps > 0) {
        const long long m = std::min(nsteps, std::max(1LL, L->ref_next - L->steps));
        goc_status st = enqueue_run(L, m);
        if (st != GOC_OK) return st;
        nsteps -= m;
        if ((st = ref_maybe_refresh(L)) != GOC_OK) return st;
    }
    return GOC_OK;
}

static goc_status enqueue_run(goc_lattice *L, long long nsteps) {
    if (L->fresh && nsteps > 0) {   // first step after initialisation: no streaming of f^0
        goc_status st = launch_one(L, nullptr);
        if (st != GOC_OK) return st;
        nsteps--;
    }
    {
        goc_status st = autotune(L, &nsteps);
        if (st != GOC_OK) return st;
    }
    if (nsteps > kGraphSteps) {
        goc_status st = ensure_graph(L);
        if (st != GOC_OK) return st;
        if (L->cur != L->graph_cur) {   // align the buffer parity with the captured graph
            if ((st = launch_one(L, nullptr)) != GOC_OK) return st;
            nsteps--;
        }
        while (nsteps >= kGraphSteps) {
            CU(cudaGraphLaunch(L->graph, L->stream));
            L->steps += kGraphSteps;   // kGraphSteps is even: the current buffer is unchanged
            nsteps -= kGraphSteps;
        }
    }
    for (long long s = 0; s < nsteps; s++) {
        goc_status st = launch_one(L, nullptr);
        if (st != GOC_OK) return st;
    }
    return GOC_OK;
}

goc_status goc_sync(goc_lattice *L) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    CU(cudaStreamSynchronize(L->stream));
    return device_status(L);
}

long long goc_steps_done(const goc_lattice *L) { return L ? L->steps : -1; }

goc_status goc_launch_config(const goc_lattice *L, int *dynamic_tiles, int *pdl, int *tuned) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (dynamic_tiles) *dynamic_tiles = L->cfg_dynamic;
    if (pdl) *pdl = L->cfg_pdl;
    if (tuned) *tuned = L->tuned ? 1 : 0;
    return GOC_OK;
}

goc_status goc_launch_grid(const goc_lattice *L, int *balanced) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (balanced) *balanced = L->cfg_balanced;
    return GOC_OK;
}

goc_status goc_tile_height(const goc_lattice *L, int *rows) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (rows) *rows = tile_rows_apply(L) ? 8 * L->cfg_rows : TY;
    return GOC_OK;
}

goc_status goc_set_tile_height(goc_lattice *L, int rows) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (rows != 8 && rows != 16) return fail(GOC_EINVAL, "the tile height must be 8 or 16 rows");
    if (rows == 16 && !tile_rows_apply(L))
        return fail(GOC_EINVAL, "16-row tiles are for straight grids with the central-moment collision");
    L->cfg_rows = rows / 8;
    L->tuned = true;
    if (L->graph) {   // captured under another configuration
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    return GOC_OK;
}

goc_status goc_set_launch_grid(goc_lattice *L, int balanced) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (balanced != 0 && balanced != 1) return fail(GOC_EINVAL, "balanced must be 0 or 1");
    L->cfg_balanced = balanced;
    L->tuned = true;
    if (L->graph) {   // captured under another configuration
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    return GOC_OK;
}

goc_status goc_set_launch_config(goc_lattice *L, int dynamic_tiles, int pdl) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if ((dynamic_tiles != 0 && dynamic_tiles != 1) || (pdl != 0 && pdl != 1))
        return fail(GOC_EINVAL, "dynamic_tiles and pdl must be 0 or 1");
    L->cfg_dynamic = dynamic_tiles;
    L->cfg_pdl = pdl;
    L->tuned = true;
    if (L->graph) {   // captured under another configuration
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    return GOC_OK;
}

goc_status goc_footprint(const goc_lattice *L, long long *nodes, long long *bytes) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (nodes) *nodes = (long long)L->nx * L->ny;
    if (bytes) *bytes = (long long)L->device_bytes + (L->mom ? 0 : 0);
    return GOC_OK;
}

double goc_bytes_per_node(const goc_lattice *L) {
    if (!L) return 0.0;
    const double es = (double)elem_size(L->storage);
    if (L->scheme == 1) return 2.0 * 9.0 * es;          // populations only, read + write
    if (L->aa)   // fields pass: populations, force read, fields written; collision pass: populations, force
                 // and fields read, populations and force written
        return 33.0 * es + 24.0 + (L->mhd.enabled ? 2.0 * 10.0 * es : 0.0) + 4.0 * 7.0 / L->ny + 4.0 * 7.0 / L->nx;
    double b = 2.0 * (9.0 + 2.0) * es;                  // populations + stored force, read + write
    if (L->mhd.enabled) b += 2.0 * 10.0 * es;           // MIE populations
    if (L->sp.curv == 2) return b + 4.0 * 10.0;         // node-table metric: 10 FP32 values per node
    b += 4.0 * (L->sp.curv ? 8.0 : 7.0) / L->ny + 4.0 * 7.0 / L->nx;   // per-axis tables amortised over the lattice
    return b;
}

goc_status goc_moments(goc_lattice *L, int cartesian, double *rho, double *u1, double *u2,
                       double *b1, double *b2) {
    TraceRange trace_("goc_moments");
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    const bool rotate = cartesian && L->map.kind[0] == GOC_MAP_ANNULUS;
    if (cartesian && L->map.kind[0] == GOC_MAP_TABLE)
        return fail(GOC_EUNSUPPORTED, "a TABLE map carries no coordinates: Cartesian components are unavailable");
    goc_status st = moments_to_device(L);
    if (st != GOC_OK) return st;
    const long long N = (long long)L->nx * L->ny;
    double *outs[5] = {rho, u1, u2, b1, b2};
    // the annulus rotates both components of a vector: fetch the pair whole
    std::vector<double> tmp;
    if (rotate) tmp.assign(4 * (size_t)N, 0.0);
    for (int k = 0; k < 5; k++) {
        double *dst = outs[k];
        if (rotate && k >= 1) dst = tmp.data() + (k - 1) * N;
        if (dst) CU(cudaMemcpyAsync(dst, L->mom + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    }
    CU(cudaStreamSynchronize(L->stream));
    const goc_status fs = device_status(L);   // the fields are returned either way
    if (rotate) {   // Eq. vectormapping on the annular sector: xi1 radial, xi2 azimuthal at
                    // phi = (pi/sectors)(2 xi2/ny - 1), periodic nodes at xi2 = j
        const double PI = 3.14159265358979323846;
        for (int j = 0; j < L->ny; j++) {
            const double phi = PI / L->map.sectors * (2.0 * j / L->ny - 1.0), c = std::cos(phi), s = std::sin(phi);
            for (int i = 0; i < L->nx; i++) {
                const long long n = (long long)j * L->nx + i;
                for (int v = 0; v < 2; v++) {
                    const double vr = tmp[(2 * v) * N + n], vp = tmp[(2 * v + 1) * N + n];
                    double *ox = outs[1 + 2 * v], *oy = outs[2 + 2 * v];
                    if (ox) ox[n] = c * vr - s * vp;
                    if (oy) oy[n] = s * vr + c * vp;
                }
            }
        }
    }
    return fs;
}

goc_status goc_moments_device(goc_lattice *L, float *out) {
    if (!L || !out) return fail(GOC_EINVAL, "lattice and out are required");
    goc_status st = moments_to_device(L);
    if (st != GOC_OK) return st;
    const long long n = 5LL * L->nx * L->ny;
    to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, L->stream>>>(L->mom, out, n);
    CU(cudaGetLastError());
    return GOC_OK;
}

goc_status goc_diagnostics(goc_lattice *L, double *mass, double *residual_u, double *residual_b) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (mass) {
        StepParams p = params_for(L, L->cur, nullptr);
        CU(cudaMemsetAsync(L->red, 0, sizeof(double), L->stream));
        switch (L->storage) {
            case GOC_FP16_DEV: mass_kernel<__half><<<296, 256, 0, L->stream>>>(p, L->red); break;
            case GOC_BF16_DEV: mass_kernel<__nv_bfloat16><<<296, 256, 0, L->stream>>>(p, L->red); break;
            default: mass_kernel<float><<<296, 256, 0, L->stream>>>(p, L->red); break;
        }
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(mass, L->red, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        CU(cudaStreamSynchronize(L->stream));
    }
    if (residual_u) *residual_u = L->res_u;
    if (residual_b) *residual_b = L->res_b;
    return GOC_OK;
}

goc_status goc_run_until(goc_lattice *L, double tol, long long max_steps, long long *done, double *residual) {
    TraceRange trace_("goc_run_until");
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (L->slab) return fail(GOC_EUNSUPPORTED, "goc_run_until needs the whole lattice: a slab's residual is one share of it");
    if (max_steps < 0) return fail(GOC_EINVAL, "max_steps must be >= 0");
    if (!L->uout[0]) {
        for (int b = 0; b < 2; b++) {
            cudaError_t e = cudaMalloc(&L->uout[b], 4 * L->plane * sizeof(float));
            if (e != cudaSuccess) return fail(GOC_ENOMEM, "residual buffers: %s", cudaGetErrorString(e));
            L->device_bytes += 4 * L->plane * sizeof(float);
        }
    }
    long long taken = 0;
    double R = 1e300, best = 1e300;
    int h_flag = 0, stall = 0;
    const int K = std::max(2, L->check_every);
    while (taken < max_steps) {
        long long chunk = std::min<long long>(K, max_steps - taken);
        if (chunk >= 2) {
            goc_status st = goc_step(L, chunk - 2);
            if (st != GOC_OK) return st;
            if ((st = launch_one(L, L->uout[0])) != GOC_OK) return st;
            if ((st = launch_one(L, L->uout[1])) != GOC_OK) return st;
            if ((st = ref_maybe_refresh(L)) != GOC_OK) return st;
            CU(cudaMemsetAsync(L->red, 0, 4 * sizeof(double), L->stream));
            residual_kernel<<<296, 256, 0, L->stream>>>(L->uout[0], L->uout[1], L->plane, L->nx, L->ny, L->pitch, L->red);
            CU(cudaGetLastError());
            double h[4];
            CU(cudaMemcpyAsync(h, L->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
            CU(cudaMemcpyAsync(&h_flag, L->flag, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
            CU(cudaStreamSynchronize(L->stream));
            taken += chunk;
            L->res_u = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
            L->res_b = (L->mhd.enabled && h[3] > 0) ? std::sqrt(h[2] / h[3]) : 0.0;
            R = std::max(L->res_u, L->res_b);
            if (h_flag || !std::isfinite(R)) {
                if (done) *done = taken;
                if (residual) *residual = R;
                return h_flag ? flag_status(L, h_flag) : fail(GOC_EDIVERGED, "lattice diverged after %lld steps", L->steps);
            }
            if (R < tol) break;
            if (R < best) {
                best = R;
                stall = 0;
            } else if (L->plateau_checks > 0 && ++stall >= L->plateau_checks) {
                break;   // rounding floor above the tolerance
            }
        } else {
            goc_status st = goc_step(L, chunk);
            if (st != GOC_OK) return st;
            taken += chunk;
        }
    }
    if (done) *done = taken;
    if (residual) *residual = R;
    return GOC_OK;
}

goc_status goc_get_state(goc_lattice *L, void *buf, size_t *bytes) {
    if (!L || !bytes) return fail(GOC_EINVAL, "lattice and bytes are required");
    const size_t es = elem_size(L->storage);
    const size_t nf = 9 * L->plane * es, nF = 2 * L->plane * es, ng = L->mhd.enabled ? 10 * L->plane * es : 0;
    const size_t nr = L->ref64 ? 3 * (size_t)L->ny * sizeof(double) : 0;   // per-row storage reference
    const size_t total = 64 + nf + nF + ng + nr;
    if (!buf) {
        *bytes = total;
        return GOC_OK;
    }
    if (*bytes < total) return fail(GOC_EINVAL, "buffer too small (%zu < %zu)", *bytes, total);
    char *c = static_cast<char *>(buf);
    // hdr[7]: 1 the state is f^0 (the next step reads it in place); in-place
    // lattices add 2, and 4 when the populations are in the layout of odd
    // parity (see goc_aa.cuh)
    long long hdr[8] = {0x474f434c4154ll, L->nx, L->ny, L->storage, L->mhd.enabled, L->steps, (long long)total,
                        (L->fresh ? 1 : 0) | (L->aa ? 2 : 0) | (L->aa && L->cur ? 4 : 0)};
    std::memcpy(c, hdr, sizeof hdr);
    CU(cudaMemcpyAsync(c + 64, L->f[L->cur], nf, cudaMemcpyDeviceToHost, L->stream));
    CU(cudaMemcpyAsync(c + 64 + nf, L->F[L->cur], nF, cudaMemcpyDeviceToHost, L->stream));
    if (ng) CU(cudaMemcpyAsync(c + 64 + nf + nF, L->g[L->cur], ng, cudaMemcpyDeviceToHost, L->stream));
    if (nr) CU(cudaMemcpyAsync(c + 64 + nf + nF + ng, L->ref64, nr, cudaMemcpyDeviceToHost, L->stream));
    CU(cudaStreamSynchronize(L->stream));
    *bytes = total;
    return GOC_OK;
}

goc_status goc_set_state(goc_lattice *L, const void *buf, size_t bytes) {
    if (!L || !buf) return fail(GOC_EINVAL, "lattice and buf are required");
    const char *c = static_cast<const char *>(buf);
    long long hdr[8];
    if (bytes < sizeof hdr) return fail(GOC_EINVAL, "state buffer too small");
    std::memcpy(hdr, c, sizeof hdr);
    const size_t es = elem_size(L->storage);
    const size_t nf = 9 * L->plane * es, nF = 2 * L->plane * es, ng = L->mhd.enabled ? 10 * L->plane * es : 0;
    const size_t nr = L->ref64 ? 3 * (size_t)L->ny * sizeof(double) : 0;
    if (hdr[0] != 0x474f434c4154ll || hdr[1] != L->nx || hdr[2] != L->ny || hdr[3] != L->storage ||
        hdr[4] != L->mhd.enabled || (size_t)hdr[6] != 64 + nf + nF + ng + nr || bytes < 64 + nf + nF + ng + nr ||
        ((hdr[7] & 2) != 0) != L->aa)
        return fail(GOC_EINVAL, "state does not match this lattice");
    if (L->aa) L->cur = (hdr[7] & 4) ? 1 : 0;   // the layout of the saved populations
    CU(cudaMemcpyAsync(L->f[L->cur], c + 64, nf, cudaMemcpyHostToDevice, L->stream));
    CU(cudaMemcpyAsync(L->F[L->cur], c + 64 + nf, nF, cudaMemcpyHostToDevice, L->stream));
    if (ng) CU(cudaMemcpyAsync(L->g[L->cur], c + 64 + nf + nF, ng, cudaMemcpyHostToDevice, L->stream));
    if (nr) {
        CU(cudaMemcpyAsync(L->ref64, c + 64 + nf + nF + ng, nr, cudaMemcpyHostToDevice, L->stream));
        goc_status st = ref_tables(L, L->ref64);
        if (st != GOC_OK) return st;
    }
    const unsigned step = (unsigned)hdr[5];   // the stochastic-rounding stream continues from the saved step
    CU(cudaMemcpyAsync(L->flag + 2 + L->cur, &step, sizeof(unsigned), cudaMemcpyHostToDevice, L->stream));
    CU(cudaMemsetAsync(L->flag, 0, sizeof(int), L->stream));   // a restored state starts with a clear status
    CU(cudaStreamSynchronize(L->stream));
    if (L->hflag) *L->hflag = 0;
    L->steps = hdr[5];
    L->fresh = (hdr[7] & 1) != 0;
    if (L->ref_every > 0) L->ref_next = (L->steps / L->ref_every + 1) * L->ref_every;
    return GOC_OK;
}


// ---- slab decomposition of one lattice along xi2 --------------------------

goc_status goc_create_slab(const goc_grid *grid, const goc_map *map, const goc_flow *flow, const goc_mhd *mhd,
                           const goc_exec *exec, int row_begin, int row_end, goc_lattice **out) {
    if (!out) return fail(GOC_EINVAL, "out is NULL");
    *out = nullptr;
    goc_status st = validate(grid, map);
    if (st != GOC_OK) return st;
    if (map->kind[0] == GOC_MAP_ANNULUS || map->kind[0] == GOC_MAP_TABLE)
        return fail(GOC_EUNSUPPORTED, "slabs take per-axis maps (straight grids)");
    if (exec && exec->streaming != 0) return fail(GOC_EUNSUPPORTED, "slabs keep two population buffers");
    const bool per = grid->bc[2] == GOC_BC_PERIODIC;
    if (!(0 <= row_begin && row_begin + kSlabGhost <= row_end && row_end <= grid->ny))
        return fail(GOC_EINVAL, "slab rows [%d, %d) of %d: need 0 <= begin, end - begin >= %d, end <= ny",
                    row_begin, row_end, grid->ny, kSlabGhost);
    if (per && row_end - row_begin > grid->ny - kSlabGhost)
        return fail(GOC_EINVAL, "on a periodic xi2 axis a slab leaves at least %d rows to its neighbours", kSlabGhost);
    SlabPlan plan;
    plan.global = grid;
    plan.r0 = row_begin;
    plan.r1 = row_end;
    plan.glo = (per || row_begin > 0) ? kSlabGhost : 0;
    plan.ghi = (per || row_end < grid->ny) ? kSlabGhost : 0;
    goc_grid local = *grid;
    local.ny = (row_end - row_begin) + plan.glo + plan.ghi;
    for (int s = 2; s < 4; s++) {   // an internal cut is a wall of the local lattice (only ghost rows see it)
        const bool cut = s == 2 ? plan.glo > 0 : plan.ghi > 0;
        if (!cut) continue;
        local.bc[s] = GOC_BC_WALL;
        local.wall_u[s] = 0.0;
        local.wall_b[s][0] = local.wall_b[s][1] = 0.0;
    }
    if (per) local.bc[2] = local.bc[3] = GOC_BC_WALL;
    return create_impl(&local, map, flow, mhd, exec, &plan, out);
}

goc_status goc_slab_info(const goc_lattice *L, int *row_begin, int *row_end, int *ghost_lo, int *ghost_hi) {
    if (!L) return fail(GOC_EINVAL, "lattice is NULL");
    if (row_begin) *row_begin = L->slab ? L->slab_r0 : 0;
    if (row_end) *row_end = L->slab ? L->slab_r1 : L->ny;
    if (ghost_lo) *ghost_lo = L->slab_glo;
    if (ghost_hi) *ghost_hi = L->slab_ghi;
    return GOC_OK;
}

static int slab_planes(const goc_lattice *L) { return 11 + (L->mhd.enabled ? 10 : 0); }
static size_t slab_plane_bytes(const goc_lattice *L) {
    return ((size_t)slab_planes(L) * kSlabGhost * L->nx * elem_size(L->storage) + 7) / 8 * 8;
}

long long goc_slab_halo_bytes(const goc_lattice *L) {
    if (!L || !L->slab) return 0;
    return (long long)(slab_plane_bytes(L) + (L->ref64 ? 3 * kSlabGhost * sizeof(double) : 0));
}

// rows [row, row + 2) of the current state to (unpack = 0) or from (1) msg
static goc_status slab_move(goc_lattice *L, void *msg, int row, int unpack) {
    StepParams p = params_for(L, L->cur, nullptr);
    const dim3 grid((L->nx + 127) / 128, kSlabGhost, slab_planes(L));
    switch (L->storage) {
        case GOC_FP16_DEV: halo_kernel<__half><<<grid, 128, 0, L->stream>>>(p, static_cast<__half *>(msg), row, unpack); break;
        case GOC_BF16_DEV:
            halo_kernel<__nv_bfloat16><<<grid, 128, 0, L->stream>>>(p, static_cast<__nv_bfloat16 *>(msg), row, unpack);
            break;
        default: halo_kernel<float><<<grid, 128, 0, L->stream>>>(p, static_cast<float *>(msg), row, unpack); break;
    }
    CU(cudaGetLastError());
    if (L->ref64) {
        halo_ref_kernel<<<1, 32, 0, L->stream>>>(L->ref64, L->ny, reinterpret_cast<double *>(static_cast<char *>(msg) +
                                                                                             slab_plane_bytes(L)),
                                                 row, unpack);
        CU(cudaGetLastError());
    }
    return GOC_OK;
}

goc_status goc_slab_pack(goc_lattice *L, void *send_lo, void *send_hi) {
    if (!L || !L->slab) return fail(GOC_EINVAL, "not a slab");
    const int own0 = L->slab_glo, own1 = L->ny - L->slab_ghi;
    goc_status st = GOC_OK;
    if (send_lo && L->slab_glo) st = slab_move(L, send_lo, own0, 0);
    if (st == GOC_OK && send_hi && L->slab_ghi) st = slab_move(L, send_hi, own1 - kSlabGhost, 0);
    return st;
}

goc_status goc_slab_unpack(goc_lattice *L, const void *recv_lo, const void *recv_hi) {
    if (!L || !L->slab) return fail(GOC_EINVAL, "not a slab");
    const int own1 = L->ny - L->slab_ghi;
    goc_status st = GOC_OK;
    if (recv_lo && L->slab_glo) st = slab_move(L, const_cast<void *>(recv_lo), 0, 1);
    if (st == GOC_OK && recv_hi && L->slab_ghi) st = slab_move(L, const_cast<void *>(recv_hi), own1, 1);
    if (st == GOC_OK && L->ref64) st = ref_tables(L, L->ref64);   // the ghost rows' storage reference changed
    return st;
}

}  // extern "C"

// ============================================================================
// Batched execution: all resident lattices advance together, one persistent
// launch per time step and storage type, captured in a CUDA graph.
// ============================================================================
struct goc_batch {
    long long budget = 0, used = 0;
    int max_lat = 0;
    int storage = GOC_FP32;
    int rounding = 0;
    int reference_every = 0;      // goc_exec.reference_every of the members
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<goc_lattice *> slots;
    std::vector<long long> bytes;
    bool dirty = true;
    // Members are grouped by storage type and MIE on/off (one kernel each), and
    // each group is cut into sets whose state fits in L2 together; within a
    // graph chunk each set runs all its steps before the next set starts, so a
    // set's populations stay L2-resident for the whole chunk.
    struct Group {
        int storage = 0, mhd = 0, geom = 0, n = 0, total = 0, grid = 0, stage_bytes = 0;
        std::vector<int> members;      // at most kBatchMax slots
        std::vector<BatchArgs> args;   // launch arguments: parity 0, parity 1, first step after a rebuild,
                                       // then parity p with snapshot u: 3 + 2 p + u
        CUtensorMap *maps = nullptr;   // device [2 parities][n][3]
        int *ctr = nullptr;            // device [2]: work-item counters by step parity
    };
    std::vector<Group> groups;
    long long phase = 0;
    bool first_pending = false;   // next launch uses the first-step parameters (fresh members read in place)
    cudaGraphExec_t graph = nullptr;
    std::vector<char> check;      // per slot: record successive fields for the residual
    bool any_check = false;
};

namespace {

constexpr int kBatchGraphSteps = 32;

long long estimate_bytes(const goc_grid *grid, const goc_map *map, const goc_mhd *mhd, int storage) {
    const long long pitch = (grid->nx + 31) / 32 * 32;
    const long long plane = pitch * grid->ny;
    const long long es = (long long)elem_size(storage);
    long long b = 2 * (9 + 2) * plane * es;
    if (mhd && mhd->enabled) b += 2 * 10 * plane * es;
    b += 8LL * 4 * (grid->nx + grid->ny) + 32LL * (grid->nx + grid->ny + 4) + 128;
    b += 36LL * (grid->nx + grid->ny);   // spare table row and per-index metric records
    if (map && map->kind[0] == GOC_MAP_TABLE)   // node-table metric planes and wall factors
        b += (10 * plane + 8LL * std::max(grid->nx, grid->ny)) * 4;
    if (storage != GOC_FP32) b += 6LL * 8 * grid->ny + 7LL * 4 * grid->ny;   // per-row storage reference
    return b;
}

void free_groups(goc_batch *B) {
    for (auto &g : B->groups) {
        if (g.maps) cudaFree(g.maps);
        if (g.ctr) cudaFree(g.ctr);
    }
    B->groups.clear();
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
}

// bytes of lattice state per set: one set per kernel type, or with
// GOC_BATCH_L2_SETS=1 sets of three quarters of the L2 size (measured slower on
// the 64-lattice batch: the step is instruction-bound, and smaller launches
// add tails)
long long l2_set_bytes(int device) {
    const char *e = std::getenv("GOC_BATCH_L2_SETS");
    if (!e || std::atoi(e) == 0) return (1LL << 62);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    return l2 > 0 ? 3LL * l2 / 4 : (1LL << 62);
}


// Kernel type of a batch group: storage (3) x MIE (2) x grid kind (straight,
// annular sector, node table); one batch kernel instantiation each.
int batch_key(int storage, int mhd, int geom) { return (geom * 3 + storage) * 2 + mhd; }

goc_status rebuild(goc_batch *B) {
    free_groups(B);
    const long long cap = l2_set_bytes(B->device);
    for (int key = 0; key < 18; key++) {   // kernel type (batch_key); launches of <= kBatchMax lattices
        long long used = 0;
        for (int k = 0; k < (int)B->slots.size(); k++) {
            goc_lattice *L = B->slots[k];
            if (!L || batch_key(L->storage, L->mhd.enabled ? 1 : 0, L->sp.curv) != key) continue;
            if (B->groups.empty() ||
                batch_key(B->groups.back().storage, B->groups.back().mhd, B->groups.back().geom) != key ||
                (int)B->groups.back().members.size() == kBatchMax ||
                (used + B->bytes[k] > cap && !B->groups.back().members.empty())) {
                goc_batch::Group g;
                g.mhd = key % 2;
                g.storage = (key / 2) % 3;
                g.geom = key / 6;
                B->groups.push_back(std::move(g));
                used = 0;
            }
            B->groups.back().members.push_back(k);
            used += B->bytes[k];
        }
    }
    for (auto &g : B->groups) {
        g.n = (int)g.members.size();
        std::vector<int> tiles(g.n);
        g.total = 0;
        for (int m = 0; m < g.n; m++) {
            const goc_lattice *L = B->slots[g.members[m]];
            tiles[m] = ((L->nx + TX - 1) / TX) * ((L->ny + TY - 1) / TY);
            g.total += tiles[m];
        }
        int capacity = 0;   // resident blocks of this kernel on the device
        capacity = g.storage == GOC_FP16_DEV   ? batch_grid_t<__half>(g.mhd, g.geom, &g.stage_bytes)
                   : g.storage == GOC_BF16_DEV ? batch_grid_t<__nv_bfloat16>(g.mhd, g.geom, &g.stage_bytes)
                                               : batch_grid_t<float>(g.mhd, g.geom, &g.stage_bytes);
        g.grid = std::min(g.total, capacity);   // persistent blocks taking tiles from the counter
        g.args.assign(7, BatchArgs{});
        CU(cudaMalloc(&g.ctr, 2 * sizeof(int)));
        CU(cudaMemsetAsync(g.ctr, 0, 2 * sizeof(int), B->stream));
        for (int v = 0; v < 7; v++) {
            auto &a = g.args[v];
            a.n = g.n;
            a.toff[0] = 0;
            for (int m = 0; m < g.n; m++) a.toff[m + 1] = a.toff[m] + tiles[m];
            a.parity = v == 1 ? 1 : (v >= 3 ? (v - 3) / 2 : 0);
            a.ctr = g.ctr;
        }
        std::vector<CUtensorMap> hm(2 * 3 * g.n);
        for (int m = 0; m < g.n; m++) {
            const goc_lattice *L = B->slots[g.members[m]];
            for (int par = 0; par < 2; par++) {
                const int src = L->cur ^ par;
                hm[(par * g.n + m) * 3 + 0] = L->tmf[src];
                hm[(par * g.n + m) * 3 + 1] = L->tmF[src];
                hm[(par * g.n + m) * 3 + 2] = L->mhd.enabled ? L->tmg[src] : L->tmf[src];
            }
        }
        CU(cudaMalloc(&g.maps, hm.size() * sizeof(CUtensorMap)));
        CU(cudaMemcpyAsync(g.maps, hm.data(), hm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, B->stream));
        for (int v = 0; v < 7; v++) {   // variant v reads the buffers of parity 0 (v = 0, 2), 1 (v = 1), or 3 + 2 p + u
            const int par = v == 1 ? 1 : (v >= 3 ? (v - 3) / 2 : 0);
            g.args[v].maps = g.maps + par * 3 * g.n;
        }
        for (int m = 0; m < g.n; m++) {
            const int slot = g.members[m];
            goc_lattice *L = B->slots[slot];
            g.args[0].p[m] = params_for(L, L->cur, nullptr);
            g.args[1].p[m] = params_for(L, L->cur ^ 1, nullptr);
            g.args[2].p[m] = g.args[0].p[m];
            g.args[2].p[m].nopull = L->fresh ? 1 : 0;
            for (int par = 0; par < 2; par++)
                for (int u = 0; u < 2; u++)
                    g.args[3 + 2 * par + u].p[m] = params_for(L, L->cur ^ par, B->check[slot] ? L->uout[u] : nullptr);
        }
    }
    CU(cudaStreamSynchronize(B->stream));
    B->phase = 0;
    B->dirty = false;
    B->first_pending = true;
    return GOC_OK;
}

goc_status batch_launch(goc_batch *B, cudaStream_t st, long long s, bool first = false, int snapshot = -1,
                        int only = -1) {
    for (int gi = 0; gi < (int)B->groups.size(); gi++) {
        if (only >= 0 && gi != only) continue;
        auto &g = B->groups[gi];
        if (!g.n) continue;
        const int par = (int)((B->phase + s) & 1);
        const int which = first ? 2 : (snapshot >= 0 ? 3 + 2 * par + snapshot : par);
        const BatchArgs &a = g.args[which];
        const size_t smem = 2 * (size_t)g.stage_bytes;
        const dim3 gd(g.grid), bd(TX, TYT);
        cudaError_t e;
        e = g.storage == GOC_FP16_DEV   ? batch_launch_t<__half>(g.mhd, g.geom, gd, bd, smem, st, a)
            : g.storage == GOC_BF16_DEV ? batch_launch_t<__nv_bfloat16>(g.mhd, g.geom, gd, bd, smem, st, a)
                                        : batch_launch_t<float>(g.mhd, g.geom, gd, bd, smem, st, a);
        CU(e);
        CU(cudaGetLastError());
    }
    return GOC_OK;
}

}  // namespace

extern "C" {

goc_status goc_batch_create(long long hbm_budget_bytes, int max_lattices, const goc_exec *exec, goc_batch **out) {
    if (!out) return fail(GOC_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_lattices <= 0) return fail(GOC_EINVAL, "budget and max_lattices must be > 0");
    if (exec && exec->streaming != 0) return fail(GOC_EUNSUPPORTED, "batched lattices keep two population buffers");
    goc_batch *B = new (std::nothrow) goc_batch();
    if (!B) return fail(GOC_ENOMEM, "host allocation failed");
    B->budget = hbm_budget_bytes;
    B->max_lat = max_lattices;
    if (exec) {
        B->storage = exec->storage;
        B->rounding = exec->rounding;
        B->reference_every = exec->reference_every;
        B->stream = (cudaStream_t)exec->cuda_stream;
        if (exec->device >= 0) cudaSetDevice(exec->device);
    }
    cudaGetDevice(&B->device);
    B->slots.assign(max_lattices, nullptr);
    B->bytes.assign(max_lattices, 0);
    B->check.assign(max_lattices, 0);
    *out = B;
    return GOC_OK;
}

void goc_batch_destroy(goc_batch *B) {
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    for (auto *L : B->slots)
        if (L) free_lattice(L);
    free_groups(B);
    delete B;
}

goc_status goc_batch_add(goc_batch *B, const goc_grid *grid, const goc_map *map, const goc_flow *flow,
                         const goc_mhd *mhd, int storage, int *slot) {
    if (!B || !slot) return fail(GOC_EINVAL, "batch and slot are required");
    *slot = -1;
    if (!grid) return fail(GOC_EINVAL, "grid is required");
    int free_slot = -1;
    for (int k = 0; k < B->max_lat; k++)
        if (!B->slots[k]) {
            free_slot = k;
            break;
        }
    if (free_slot < 0) return fail(GOC_EBUSY, "batch is full (%d lattices)", B->max_lat);
    const long long need = estimate_bytes(grid, map, mhd, storage);
    if (B->used + need > B->budget)
        return fail(GOC_EBUSY, "HBM budget exhausted (%lld + %lld > %lld bytes)", B->used, need, B->budget);
    goc_exec ex;
    std::memset(&ex, 0, sizeof ex);
    ex.storage = storage;
    ex.cuda_stream = B->stream;
    ex.device = -1;
    ex.rounding = B->rounding;
    ex.reference_every = B->reference_every;
    goc_lattice *L = nullptr;
    goc_status st = goc_create(grid, map, flow, mhd, &ex, &L);
    if (st != GOC_OK) return st;
    L->in_batch = true;
    B->slots[free_slot] = L;
    B->bytes[free_slot] = (long long)L->device_bytes;
    B->used += (long long)L->device_bytes;
    B->dirty = true;
    *slot = free_slot;
    return GOC_OK;
}

goc_status goc_batch_remove(goc_batch *B, int slot) {
    if (!B || slot < 0 || slot >= B->max_lat || !B->slots[slot]) return fail(GOC_EINVAL, "no lattice in slot %d", slot);
    cudaStreamSynchronize(B->stream);
    B->used -= B->bytes[slot];
    free_lattice(B->slots[slot]);
    B->slots[slot] = nullptr;
    B->bytes[slot] = 0;
    B->check[slot] = 0;
    B->any_check = false;
    for (char c : B->check) B->any_check = B->any_check || c;
    B->dirty = true;
    return GOC_OK;
}

goc_status goc_batch_step(goc_batch *B, long long nsteps) {
    TraceRange trace_("goc_batch_step");
    if (!B) return fail(GOC_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(GOC_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return GOC_OK;
    if (B->dirty) {
        goc_status st = rebuild(B);
        if (st != GOC_OK) return st;
    }
    bool any = false;
    for (auto &g : B->groups) any = any || g.n > 0;
    if (!any) return GOC_OK;
    if (B->first_pending) {   // first step after a rebuild (parity 0, fresh members unstreamed)
        goc_status st = batch_launch(B, B->stream, 0, true);
        if (st != GOC_OK) return st;
        B->first_pending = false;
        B->phase += 1;
        for (auto *L : B->slots)
            if (L) {
                L->steps += 1;
                L->cur ^= 1;
                L->fresh = false;
                L->queues_dirty = true;
            }
        if (--nsteps == 0) return GOC_OK;
    }
    // with residual checks the last two steps record successive fields
    const int tail = (B->any_check && nsteps >= 2) ? 2 : 0;
    long long left = nsteps - tail;
    auto single = [&]() -> goc_status {
        goc_status st = batch_launch(B, B->stream, 0);
        B->phase += 1;
        return st;
    };
    if (left >= kBatchGraphSteps && (B->phase & 1)) {   // the graph starts on an even phase
        goc_status st = single();
        if (st != GOC_OK) return st;
        left--;
    }
    if (left >= kBatchGraphSteps) {
        if (!B->graph) {
            cudaStream_t cs;
            CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t gr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            goc_status st = GOC_OK;
            // set-major order: each L2-sized set advances all steps of the chunk in turn
            for (int gi = 0; gi < (int)B->groups.size() && st == GOC_OK && e == cudaSuccess; gi++)
                for (int k = 0; k < kBatchGraphSteps && st == GOC_OK; k++) st = batch_launch(B, cs, k, false, -1, gi);
            if (e == cudaSuccess) e = cudaStreamEndCapture(cs, &gr);
            cudaStreamDestroy(cs);
            if (st != GOC_OK) return st;
            if (e != cudaSuccess) return fail(GOC_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&B->graph, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) {
                B->graph = nullptr;
                return fail(GOC_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
            }
        }
        while (left >= kBatchGraphSteps) {
            CU(cudaGraphLaunch(B->graph, B->stream));
            B->phase += kBatchGraphSteps;
            left -= kBatchGraphSteps;
        }
    }
    while (left > 0) {
        goc_status st = single();
        if (st != GOC_OK) return st;
        left--;
    }
    for (int u = 0; u < tail; u++) {
        goc_status st = batch_launch(B, B->stream, 0, false, u);
        if (st != GOC_OK) return st;
        B->phase += 1;
    }
    for (auto *L : B->slots)
        if (L) {
            L->steps += nsteps;
            L->cur ^= (int)(nsteps & 1);
            L->queues_dirty = true;
            // per-row storage reference of 16-bit members: refreshed at the end of
            // the call in which its step count reaches the next refresh point
            goc_status st = ref_maybe_refresh(L);
            if (st != GOC_OK) return st;
        }
    if (tail) {   // residual sums of the checked lattices (read by goc_batch_residual)
        for (int k = 0; k < B->max_lat; k++) {
            goc_lattice *L = B->slots[k];
            if (!L || !B->check[k]) continue;
            CU(cudaMemsetAsync(L->red + 4, 0, 4 * sizeof(double), B->stream));
            residual_kernel<<<148, 256, 0, B->stream>>>(L->uout[0], L->uout[1], L->plane, L->nx, L->ny, L->pitch,
                                                        L->red + 4);
            CU(cudaGetLastError());
            L->res_pending = true;
        }
    }
    return GOC_OK;
}

goc_status goc_batch_check(goc_batch *B, int slot, int on) {
    if (!B || slot < 0 || slot >= B->max_lat || !B->slots[slot]) return fail(GOC_EINVAL, "no lattice in slot %d", slot);
    goc_lattice *L = B->slots[slot];
    if (on && !L->uout[0]) {
        for (int b = 0; b < 2; b++) {
            cudaError_t e = cudaMalloc(&L->uout[b], 4 * L->plane * sizeof(float));
            if (e != cudaSuccess) return fail(GOC_ENOMEM, "residual buffers: %s", cudaGetErrorString(e));
            L->device_bytes += 4 * L->plane * sizeof(float);
            B->used += 4 * L->plane * sizeof(float);
            B->bytes[slot] += 4 * L->plane * sizeof(float);
        }
    }
    B->check[slot] = on ? 1 : 0;
    B->any_check = false;
    for (char c : B->check) B->any_check = B->any_check || c;
    B->dirty = true;
    return GOC_OK;
}

goc_status goc_batch_residual(goc_batch *B, int slot, double *residual_u, double *residual_b) {
    if (!B || slot < 0 || slot >= B->max_lat || !B->slots[slot]) return fail(GOC_EINVAL, "no lattice in slot %d", slot);
    goc_lattice *L = B->slots[slot];
    if (L->res_pending) {
        double h[4];
        int flag = 0;
        CU(cudaMemcpyAsync(h, L->red + 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
        CU(cudaMemcpyAsync(&flag, L->flag, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
        CU(cudaStreamSynchronize(B->stream));
        L->res_u = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
        L->res_b = (L->mhd.enabled && h[3] > 0) ? std::sqrt(h[2] / h[3]) : 0.0;
        L->res_pending = false;
        if (flag || !std::isfinite(L->res_u) || !std::isfinite(L->res_b)) {
            if (residual_u) *residual_u = L->res_u;
            if (residual_b) *residual_b = L->res_b;
            if (flag == 2) return flag_status(L, flag);
            return fail(GOC_EDIVERGED, "lattice in slot %d diverged", slot);
        }
    }
    if (residual_u) *residual_u = L->res_u;
    if (residual_b) *residual_b = L->res_b;
    return GOC_OK;
}

goc_status goc_batch_lattice(goc_batch *B, int slot, goc_lattice **lat) {
    if (!B || !lat || slot < 0 || slot >= B->max_lat || !B->slots[slot]) return fail(GOC_EINVAL, "no lattice in slot %d", slot);
    *lat = B->slots[slot];
    return GOC_OK;
}

goc_status goc_batch_usage(const goc_batch *B, long long *used, long long *budget, int *count) {
    if (!B) return fail(GOC_EINVAL, "batch is NULL");
    if (used) *used = B->used;
    if (budget) *budget = B->budget;
    if (count) {
        int c = 0;
        for (auto *L : B->slots) c += L != nullptr;
        *count = c;
    }
    return GOC_OK;
}

}  // extern "C"

// ============================================================================
// Total mass without allocating device memory.
//
// Some callers cannot call cudaMalloc when they need a diagnostic: real-time
// loops that must not stall on the allocator, and applications that hand all
// device memory to their own pool at start-up.
// goc_mass_noalloc computes what goc_diagnostics(mass) computes, but its
// scratch (one partial sum per block plus the final sum) lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.  All calls share that array: calls whose kernels
// overlap on the GPU (different streams, different threads) race on it.
// ============================================================================
#define GOC_NOALLOC_NODES_PER_BLOCK 2048   // 256 threads x 8 nodes
static_assert(GOC_NOALLOC_MAX_NODES == (long long)GOC_NOALLOC_MAX_BLOCKS * GOC_NOALLOC_NODES_PER_BLOCK,
              "node limit of goc_mass_noalloc");

static __device__ __align__(256) double g_noalloc_scratch[GOC_NOALLOC_MAX_BLOCKS + 1];

namespace {

// Per block: the sum over its (up to 2048) nodes of sum_a f, written to
// partial[blockIdx.x] in a fixed order (no atomics, nothing to clear).
template <class S>
__global__ void mass_partial_kernel(const StepParams p, double *partial) {
    __shared__ double red[256];
    const long long N = (long long)p.nx * (p.own1 - p.own0);   // the owned rows
    const S *f = static_cast<const S *>(p.fin);
    double acc = 0.0;
    for (int k = 0; k < GOC_NOALLOC_NODES_PER_BLOCK / 256; k++) {
        const long long n = (long long)blockIdx.x * GOC_NOALLOC_NODES_PER_BLOCK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const int j = p.own0 + (int)(n / p.nx), i = (int)(n - (long long)(j - p.own0) * p.nx);
        const long long idx = (long long)j * p.pitch + i;
        double s = 0.0;
        for (int a = 0; a < 9; a++) s += (double)Store<S>::ld(f + a * p.plane + idx) * p.sf;
        acc += s + node_h1h2(p, i, j) * p.rho0;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// One block: fixed-order sum of nblocks partials into partial[GOC_NOALLOC_MAX_BLOCKS].
__global__ void mass_final_kernel(double *partial, int nblocks) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) acc += partial[b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[GOC_NOALLOC_MAX_BLOCKS] = red[0];
}

// Makes a device current for the lifetime of the guard and restores the
// caller's current device afterwards.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        ok_ = prev_ == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev_ >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev_) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;

  private:
    int prev_ = -1;
    bool ok_ = false;
};

// Device address of the scratch array, looked up once per device (the first
// call on a device does this set-up; make that call before any stream capture).
double *noalloc_scratch(goc_status *st) {
    static double *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *st = fail(GOC_ECUDA, "goc_mass_noalloc: no usable current device");
        return nullptr;
    }
    if (!addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            *st = fail(GOC_ECUDA, "goc_mass_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return nullptr;
        }
        addr[dev] = static_cast<double *>(ptr);
    }
    *st = GOC_OK;
    return addr[dev];
}

}  // namespace

extern "C" goc_status goc_mass_noalloc(goc_lattice *L, double *mass) {
    if (!L || !mass) return fail(GOC_EINVAL, "goc_mass_noalloc: lattice and mass are required");
    const long long N = (long long)L->nx * (L->sp.own1 - L->sp.own0);   // owned rows
    const long long blocks = (N + GOC_NOALLOC_NODES_PER_BLOCK - 1) / GOC_NOALLOC_NODES_PER_BLOCK;
    if (blocks > GOC_NOALLOC_MAX_BLOCKS)
        return fail(GOC_EINVAL, "goc_mass_noalloc: the lattice has %lld nodes; at most %lld are supported",
                    N, (long long)GOC_NOALLOC_MAX_BLOCKS * GOC_NOALLOC_NODES_PER_BLOCK);
    DeviceGuard guard(L->device);   // the caller's current device is restored on every return
    if (!guard.ok()) return fail(GOC_ECUDA, "goc_mass_noalloc: cannot make device %d current", L->device);
    goc_status st;
    double *scratch = noalloc_scratch(&st);
    if (!scratch) return st;
    StepParams p = params_for(L, L->cur, nullptr);
    switch (L->storage) {
        case GOC_FP16_DEV: mass_partial_kernel<__half><<<(unsigned)blocks, 256, 0, L->stream>>>(p, scratch); break;
        case GOC_BF16_DEV: mass_partial_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, L->stream>>>(p, scratch); break;
        default: mass_partial_kernel<float><<<(unsigned)blocks, 256, 0, L->stream>>>(p, scratch); break;
    }
    CU(cudaGetLastError());
    mass_final_kernel<<<1, 256, 0, L->stream>>>(scratch, (int)blocks);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(mass, scratch + GOC_NOALLOC_MAX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CU(cudaStreamSynchronize(L->stream));
    return GOC_OK;
}
