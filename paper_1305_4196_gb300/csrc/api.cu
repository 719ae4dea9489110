// api.cu - the C ABI of include/mdgb.h on top of the sm_103a kernels.
//
// Host-side orchestration only: argument checks, workspace, the cell grid,
// capacity regrowth, and the order of kernel launches on the caller's stream.
// Every arithmetic step of the hot path runs in the kernels.
#include "mdgb.h"
#include "mdgb_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

using namespace mdgb;

struct md_system {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int np = 64;
    Geometry g{};
    PairTable pt{};
    TileOffsets to{};
    double box[3] = {0, 0, 0};
    double rcut = 0, skin = 0, rl = 0, rl2 = 0, dt = 0, lim2 = 0;
    double rcut_default = 0;  // r_cut argument of md_create (pairs without a table entry)
    int precision = MD_MIXED, list_kind = MD_LIST_FULL, rebuild = MD_REBUILD_SKIN_HALF, rebuild_k = 10;
    int list_cap = 0, tile_cap = 0;
    int tile_floor = 0;  // lower bound on tile_cap after a redo (the tiles a chunk of steps grew into)
    DevState st[3]{};  // [0] the state, [1] scratch for the reorder gather, [2] snapshot for redo
    int cur = 0;       // always 0: the state lives in st[0]
    // binning scratch
    int32_t *atom_cell = nullptr, *cell_count = nullptr, *cursor = nullptr, *slot_key = nullptr,
            *slot_src = nullptr, *sorted_src = nullptr, *scan_scratch = nullptr;
    double *partials = nullptr, *out8 = nullptr;
    int nparts = 0;
    uint32_t* h_flags = nullptr;  // pinned: [0] err, [1] rebuild flag, [2..5] stats
    bool has_state = false, lists_valid = false, forces_valid = false;
    int64_t n_builds = 0, n_steps = 0, list_entries = 0;
    int max_list = 0, max_tile = 0;
    std::vector<void*> allocs;
    // launch accounting and optional event timing
    int64_t launches = 0, force_evals = 0, n_redos = 0;
    bool timing = false;
    double force_ms = 0, build_ms = 0;
    int64_t timed_force = 0, timed_build = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_force, ev_build, ev_free;
    // graph-captured time steps
    struct StepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t ev_a = nullptr, ev_b = nullptr;
        // multi-step graphs under md_set_timing: the event nodes around each step's force kernel
        std::vector<cudaGraphNode_t> ev_multi_a, ev_multi_b;
    };
    cudaStream_t cap_stream = nullptr;
    StepGraph g_first, g_mid;
    // full-list mixed path: force kernel fused with velocity Verlet, FP32 coordinates
    // double-buffered; g_fused[closing kick only / kick-kick-drift][buffer read]
    StepGraph g_fused[2][2];
    // MULTI_STEPS kick-kick-drift steps from buffer 0 in one graph (even: back in buffer 0),
    // for md_step calls without timing events: fewer graph launches per step
    StepGraph g_multi;
    float4* xr_alt = nullptr;
    int potential = 0;       // 0: Lennard-Jones pair table; 1: TB-SMA many-body (md_set_tbsma)
    TBTable tb{};
    float* emb = nullptr;    // TB-SMA: 1/sqrt(rho) per atom (cell order)
    double* pos_alt = nullptr;  // FP64 positions of buffer 1 (x, y, z: n each)
    bool graphs_valid = false;
    int graph_tile_cap = 0, graph_list_cap = 0;
    bool graph_timing = false;
    bool use_graphs = true;  // MDGB_NO_GRAPHS=1 at md_create: host-launched steps (profilers see every kernel)
    bool no_fuse = false;    // MDGB_NO_FUSE=1 at md_create: separate force and integration kernels
    long long* d_ctrl = nullptr;  // [0] step counter, [1] builds done inside graphs
    long long* h_ctrl = nullptr;  // pinned mirror
    bool snapshot_first = true;
    int compact = 0;          // grid of the occupied-block loops of a mostly empty system (see do_build)
    bool no_compact = false;  // MDGB_NO_COMPACT=1 at md_create: one CTA per block always
    // the cell grid of a mixed-precision full-list system is chosen once, at its first build
    // (regrid_first_build); MDGB_FIT_GRID=1 at md_create keeps the r_list fit
    bool grid_decided = false;
    bool fit_grid = false;
    int64_t ncell_alloc = 0;  // cells (and 1/8 as many blocks) the cell and block arrays hold
    char msg[512] = "";
};

namespace {

int fail(md_system* s, int code, const char* fmt, ...) {
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->msg, sizeof(s->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(s, MD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

#define CKL()                                                                                      \
    do {                                                                                           \
        cudaError_t e_ = cudaGetLastError();                                                       \
        if (e_ != cudaSuccess)                                                                     \
            return fail(s, MD_ERR_CUDA, "kernel launch failed (%s:%d): %s", __FILE__, __LINE__,    \
                        cudaGetErrorString(e_));                                                   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

template <typename T>
int dalloc(md_system* s, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    CK(cudaMalloc(&q, count * sizeof(T)));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MD_OK;
}

void dfree(md_system* s, void* p) {
    if (!p) return;
    auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
    if (it != s->allocs.end()) s->allocs.erase(it);
    cudaFree(p);
}

bool mixed(const md_system* s) { return s->precision == MD_MIXED; }
bool half(const md_system* s) { return s->list_kind != MD_LIST_FULL; }
// the half list evaluated with no atomic operation (k_half_af.cu)
bool af(const md_system* s) { return s->list_kind == MD_LIST_HALF_ATOMIC_FREE; }
// shared memory of the list build / of a force launch for this system's kernels
size_t list_smem(const md_system* s, int list_cap, int tile_cap) {
    return af(s) ? af_sched_smem_bytes(tile_cap) : build_lists_smem(list_cap, tile_cap);
}
size_t fsmem(const md_system* s, int with_energy, int tile_cap) {
    return af(s) ? af_force_smem_bytes(tile_cap) : force_smem_bytes(mixed(s), half(s), with_energy, tile_cap);
}
void enqueue_lists(const md_system* s, const DevState& a, cudaStream_t st) {
    if (af(s)) launch_build_sched(a, s->g, s->to, s->rl2, s->list_cap, s->tile_cap, st);
    else launch_build_lists(a, s->g, s->to, s->rl2, s->list_cap, s->tile_cap, half(s), st);
}
// md_step runs the full-list mixed path with velocity Verlet fused into the force kernel
bool fused(const md_system* s) { return mixed(s) && !half(s) && !s->no_fuse && s->potential == 0; }
// kernels per force evaluation: 8 colour launches (half lists), two passes (TB-SMA), else one
int force_kernels(const md_system* s) { return half(s) ? 8 : (s->potential == 1 ? 2 : 1); }

// The state with its positions (FP32 cell-relative and FP64) in buffer p (0: st[0],
// 1: xr_alt and pos_alt).  Fused steps read one buffer and write the other; outside
// md_step the positions are in buffer 0.
DevState view(const md_system* s, int p) {
    DevState v = s->st[0];
    if (p) {
        v.xr = s->xr_alt;
        v.x = s->pos_alt;
        v.y = s->pos_alt + s->n;
        v.z = s->pos_alt + 2 * s->n;
    }
    return v;
}
StepOut step_out(const md_system* s, int p) {
    const DevState v = view(s, p);
    return StepOut{v.xr, v.x, v.y, v.z};
}
// Positions of buffer 1 back into buffer 0 (a chunk of fused steps that ended in buffer 1).
int positions_to_buffer0(md_system* s) {
    const size_t n = (size_t)s->n;
    const DevState& a = s->st[0];
    if (cudaMemcpyAsync(a.xr, s->xr_alt, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s->stream) ||
        cudaMemcpyAsync(a.x, s->pos_alt, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream) ||
        cudaMemcpyAsync(a.y, s->pos_alt + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream) ||
        cudaMemcpyAsync(a.z, s->pos_alt + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream))
        return fail(s, MD_ERR_CUDA, "copy of the position buffers failed");
    return MD_OK;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// List capacity for a longest list of max_list entries.  Capacity costs memory only
// (2 bytes per atom per slot), never time, and a list that outgrows it inside a chunk of
// graph-launched steps costs a redo of the chunk: half as much again, plus 32.
int list_cap_for(int max_list) { return round_up(max_list + max_list / 2 + 32, 8); }

// ---- event timing
std::pair<cudaEvent_t, cudaEvent_t> take_events(md_system* s) {
    if (!s->ev_free.empty()) {
        auto e = s->ev_free.back();
        s->ev_free.pop_back();
        return e;
    }
    std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
    cudaEventCreate(&e.first);
    cudaEventCreate(&e.second);
    return e;
}

// add the elapsed times of completed event pairs (call after a stream synchronisation)
void drain_events(md_system* s) {
    for (auto& e : s->ev_force) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
            s->force_ms += ms;
            s->timed_force++;
        }
        s->ev_free.push_back(e);
    }
    for (auto& e : s->ev_build) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
            s->build_ms += ms;
            s->timed_build++;
        }
        s->ev_free.push_back(e);
    }
    s->ev_force.clear();
    s->ev_build.clear();
}

// neighbour-list matrix for the current capacity; with keep, the current lists stay valid
// (entry k of atom i sits at the same place for every capacity)
int alloc_lists(md_system* s, int cap, bool keep = false) {
    uint16_t* nl = nullptr;
    int rc = dalloc(s, &nl, (size_t)cap * s->np);
    if (rc) return rc;
    if (keep && s->st[0].nl)
        CK(cudaMemcpyAsync(nl, s->st[0].nl, sizeof(uint16_t) * (size_t)std::min(cap, s->list_cap) * s->np,
                           cudaMemcpyDeviceToDevice, s->stream));
    dfree(s, s->st[0].nl);
    s->st[0].nl = s->st[1].nl = s->st[2].nl = nl;
    s->list_cap = cap;
    s->graphs_valid = false;
    return MD_OK;
}

int sync_flags(md_system* s) {
    CK(cudaMemcpyAsync(s->h_flags, s->st[0].err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->h_flags + 1, s->st[0].rebuild_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->h_flags + 2, s->st[0].stats, 5 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    drain_events(s);
    return MD_OK;
}

int check_err(md_system* s, uint32_t mask) {
    uint32_t e = s->h_flags[0] & mask;
    if (!e) return MD_OK;
    if (e & ERR_NONFINITE) return fail(s, MD_ERR_NONFINITE, "non-finite force or coordinate");
    if (e & ERR_ESCAPE) return fail(s, MD_ERR_NONFINITE, "an atom moved more than one box length");
    if (e & ERR_SKIN) return fail(s, MD_ERR_SKIN_VIOLATION, "an atom moved more than skin/2 between rebuilds");
    if (e & ERR_LIST_OVERFLOW) return fail(s, MD_ERR_LIST_OVERFLOW, "neighbour list overflow");
    if (e & ERR_TILE_OVERFLOW) return fail(s, MD_ERR_CELL_OVERFLOW, "tile overflow");
    if (e & ERR_CELL_DENSE)
        return fail(s, MD_ERR_CELL_OVERFLOW, "a cell above 63 atoms or a phase above 255 steps (atom-free half list)");
    return fail(s, MD_ERR_ARG, "device error 0x%x", e);
}

// ---- binning: assign, count, scan, scatter, in-cell order, gather + copy back
void enqueue_bin(md_system* s, const DevState& a, cudaStream_t st) {
    const Geometry& g = s->g;
    cudaMemsetAsync(s->cell_count, 0, sizeof(int32_t) * g.ncell, st);
    cudaMemsetAsync(s->cursor, 0, sizeof(int32_t) * g.ncell, st);
    launch_bin_assign(a, g, s->atom_cell, s->cell_count, st);
    launch_scan(s->cell_count, a.cell_start, g.ncell, s->scan_scratch, st);
    launch_scatter(a, s->atom_cell, a.cell_start, s->cursor, s->slot_key, s->slot_src, st);
    launch_cell_sort(g, a.cell_start, s->slot_key, s->slot_src, s->sorted_src, st);
    launch_gather(a, s->st[1], g, s->sorted_src, s->atom_cell, st);
    launch_classify_blocks(a, g, st);
}

int do_bin(md_system* s, int p = 0) {
    if (s->n == 0) return MD_OK;
    enqueue_bin(s, view(s, p), s->stream);
    CKL();
    s->launches += 8;
    s->lists_valid = false;
    s->forces_valid = false;
    return MD_OK;
}

// ---- list build with capacity regrowth (host-visible: reads the device counters)
void set_cut_band(md_system* s);

// Cell centres (c + 1/2) w in the kernels' cell numbering, for the current grid.
int upload_centres(md_system* s) {
    const Geometry& g = s->g;
    std::vector<double> ctr(3 * (size_t)g.ncell);
    for (int c = 0; c < g.ncell; ++c) {
        int cx, cy, cz;
        cell_coords(g, c, cx, cy, cz);
        ctr[c] = (cx + 0.5) * g.w[0];
        ctr[g.ncell + c] = (cy + 0.5) * g.w[1];
        ctr[2 * (size_t)g.ncell + c] = (cz + 0.5) * g.w[2];
    }
    for (int k = 0; k < 3; ++k) s->st[k].ncell = g.ncell;
    return cudaMemcpy(s->st[0].centre, ctr.data(), sizeof(double) * ctr.size(), cudaMemcpyHostToDevice) == cudaSuccess
               ? MD_OK
               : MD_ERR_CUDA;
}

// Cells coarser than the r_list fit on the mixed full-list path.  The force kernel runs a
// 2x2x2-cell block on 256 threads, one per own atom; at the fit grid a block of the liquid
// (rho* = 0.8442, 44 cells per side at 2,048,000 atoms) holds ~190 atoms and leaves two of
// eight warps idle until its CTA ends.  Decided once, at the first build, from the fit
// grid's binning:
//  * homogeneous (every block occupied, largest tile within 1.25x the mean): cells of width
//    w = (224 / (8 rho))^(1/3), rho = N / V, fill a block with ~224 atoms on average (7/8
//    of the threads, margin for density fluctuations);
//  * otherwise (a slab, particles in vacuum): rho is the density the average atom sees
//    (sum of squared cell counts over N, per cell volume) and the target 200 atoms, since
//    the largest tiles of such systems sit further above their mean (surfaces, a cold solid
//    that contracts) and must keep the shared memory of 5 CTAs per SM.
// Per side the smallest even count with at most that width, never more than the fit's
// count nor fewer than 6 (linear block numbering where not a multiple of 4: full lists need
// no colour classes).  *changed tells whether the grid changed (lists and graphs then need
// rebuilding); MD_ERR_CUDA if the new cell centres could not be copied to the device.
int regrid_first_build(md_system* s, int nocc, int max_tile, bool* changed) {
    *changed = false;
    if (s->grid_decided) return MD_OK;
    s->grid_decided = true;
    if (s->fit_grid || !mixed(s) || half(s) || s->potential != 0 || s->n == 0) return MD_OK;
    Geometry& g = s->g;
    const double mean_tile = 8.0 * (double)s->n / g.nblock;  // 64 of the 8 * nblock cells
    double rho, target;
    if (nocc == g.nblock && max_tile <= 1.25 * mean_tile + 1.0) {
        rho = (double)s->n / (s->box[0] * s->box[1] * s->box[2]);
        target = 224.0;
    } else {
        std::vector<int32_t> cs((size_t)g.ncell + 1);
        if (cudaMemcpy(cs.data(), s->st[0].cell_start, sizeof(int32_t) * cs.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return fail(s, MD_ERR_CUDA, "reading the cell counts for the grid choice failed");
        double sq = 0.0;
        for (int c = 0; c < g.ncell; ++c) sq += (double)(cs[c + 1] - cs[c]) * (double)(cs[c + 1] - cs[c]);
        rho = sq / (double)s->n / (g.w[0] * g.w[1] * g.w[2]);
        target = 200.0;
    }
    // never more cells than the fit grid: every cell and block array is sized for it
    int nc[3];
    bool change = false;
    for (int d = 0; d < 3; ++d) {
        nc[d] = coarse_cells(s->box[d], rho, target, g.nc[d]);
        change |= nc[d] != g.nc[d];
    }
    if (!change || (int64_t)nc[0] * nc[1] * nc[2] > s->ncell_alloc) return MD_OK;
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = nc[d];
        g.w[d] = s->box[d] / nc[d];
        g.inv_w[d] = nc[d] / s->box[d];
        for (int t = 0; t < 4; ++t) s->to.off[d][t] = (float)((t - 1.5) * g.w[d]);
    }
    set_block_layout(g);
    set_cut_band(s);
    s->graphs_valid = false;
    s->lists_valid = false;
    s->forces_valid = false;
    *changed = true;
    if (upload_centres(s) != MD_OK) return fail(s, MD_ERR_CUDA, "copying the cell centres of the new grid failed");
    return MD_OK;
}

int do_build(md_system* s, int p = 0) {
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (s->timing && s->n > 0) {
        ev = take_events(s);
        CK(cudaEventRecord(ev.first, s->stream));
    }
    int rc = do_bin(s, p);
    if (rc) return rc;
    if (s->n == 0) {
        s->lists_valid = true;
        return MD_OK;
    }
    for (int attempt = 0; attempt < 4; ++attempt) {
        const DevState a = view(s, p);
        CK(cudaMemsetAsync(a.stats, 0, 4 * sizeof(int32_t), s->stream));
        CK(cudaMemsetAsync(a.err, 0, sizeof(uint32_t), s->stream));
        if (list_smem(s, s->list_cap, s->tile_cap) > 226 * 1024)
            return fail(s, MD_ERR_CELL_OVERFLOW, "tile (%d atoms) and lists (%d) exceed shared memory",
                        s->tile_cap, s->list_cap);
        enqueue_lists(s, a, s->stream);
        CKL();
        s->launches += 1;
        if (ev.second) {
            CK(cudaEventRecord(ev.second, s->stream));
            s->ev_build.push_back(ev);
            ev = {nullptr, nullptr};
        }
        rc = sync_flags(s);
        if (rc) return rc;
        const uint32_t e = s->h_flags[0];
        const int max_list = (int)s->h_flags[2], max_tile = (int)s->h_flags[3];
        bool again = false;
        if (e & ERR_TILE_OVERFLOW) {
            // a tile never holds more than all atoms plus the dummy slot
            int cap = std::max(max_tile, std::min(round_up(max_tile + max_tile / 4 + 64, 32),
                                                  round_up((int)s->n + 1, 32)));
            if (cap > 32767) return fail(s, MD_ERR_CELL_OVERFLOW, "tile of %d atoms exceeds 15-bit indices", max_tile);
            s->tile_cap = cap;
            again = true;
        }
        if (e & ERR_LIST_OVERFLOW) {
            int cap = list_cap_for(max_list);
            if (cap > 65535) return fail(s, MD_ERR_LIST_OVERFLOW, "list of %d neighbours", max_list);
            rc = alloc_lists(s, cap);
            if (rc) return rc;
            again = true;
        }
        if (!again) {
            rc = check_err(s, ~0u);
            if (rc) return rc;
            s->max_list = max_list;
            s->max_tile = max_tile;
            uint64_t sum = (uint64_t)s->h_flags[4] | ((uint64_t)s->h_flags[5] << 32);
            s->list_entries = (int64_t)sum;
            s->n_builds++;
            s->lists_valid = true;
            // a system with a tenth or more of its blocks empty runs the full-list mixed
            // force kernel and the list builder over its occupied blocks, with a grid sized
            // for the occupied count plus headroom (more blocks later only loop further).  A
            // rebuild inside a graph keeps the grid of the last host-side build; a new grid
            // recaptures the graphs, and is only taken when the count outgrew the old one or
            // fell well below it.
            const int nocc = (int)s->h_flags[6];
            int want = 0;
            if (!s->no_compact && mixed(s) && !half(s) && 10 * (s->g.nblock - nocc) >= s->g.nblock)
                want = std::min(s->g.nblock, nocc + nocc / 8 + 152);
            if (want == 0 || s->compact == 0 || want > s->compact || 2 * want < s->compact) {
                if (want != s->compact) {
                    s->compact = want;
                    for (int k = 0; k < 3; ++k) s->st[k].compact = want;
                    s->graphs_valid = false;
                }
            }
            // keep the tile capacity close to the need (max_tile counts the dummy slot) so
            // that more CTAs fit per SM and every shared-memory layout stays within limits
            // (25 % headroom: later rebuilds inside graph-launched steps reuse this capacity)
            s->tile_cap = std::max(max_tile, std::min(round_up(max_tile + max_tile / 4 + 64, 32),
                                                      round_up((int)s->n + 1, 32)));
            s->tile_cap = std::max(s->tile_cap, s->tile_floor);
            bool changed = false;
            if ((rc = regrid_first_build(s, nocc, max_tile, &changed))) return rc;
            if (changed) {
                --s->n_builds;  // the fit grid's build is replaced
                return do_build(s, p);
            }
            return MD_OK;
        }
    }
    return fail(s, MD_ERR_LIST_OVERFLOW, "capacity regrowth did not converge");
}

void enqueue_forces(md_system* s, int with_energy, cudaStream_t st) {
    const DevState& a = s->st[0];
    if (s->potential == 1) launch_tbsma(a, s->g, s->tb, s->to, s->tile_cap, s->emb, with_energy, st);
    else if (mixed(s) && af(s)) launch_forces_half_af(a, s->g, s->pt, s->to, s->tile_cap, fs2_max_of(s->pt), with_energy, st);
    else if (mixed(s)) launch_forces_mixed(a, s->g, s->pt, s->to, s->tile_cap, half(s), with_energy, st);
    else launch_forces_fp64(a, s->g, s->pt, s->tile_cap, half(s), with_energy, st);
}

int do_forces(md_system* s, int with_energy) {
    if (s->n == 0) return MD_OK;
    const DevState& a = s->st[s->cur];
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (s->timing && !with_energy) {
        ev = take_events(s);
        CK(cudaEventRecord(ev.first, s->stream));
    }
    if (s->potential == 1) {
        if (tbsma_smem_bytes(s->tile_cap) > 226 * 1024)
            return fail(s, MD_ERR_CELL_OVERFLOW, "tile of %d atoms exceeds shared memory", s->tile_cap);
        launch_tbsma(a, s->g, s->tb, s->to, s->tile_cap, s->emb, with_energy, s->stream);
    } else if (mixed(s)) {
        if (fsmem(s, with_energy, s->tile_cap) > 226 * 1024)
            return fail(s, MD_ERR_CELL_OVERFLOW, "tile of %d atoms exceeds shared memory", s->tile_cap);
        if (af(s)) launch_forces_half_af(a, s->g, s->pt, s->to, s->tile_cap, fs2_max_of(s->pt), with_energy, s->stream);
        else launch_forces_mixed(a, s->g, s->pt, s->to, s->tile_cap, half(s), with_energy, s->stream);
    } else {
        if (force_smem_bytes(0, half(s), with_energy, s->tile_cap) > 226 * 1024)
            return fail(s, MD_ERR_CELL_OVERFLOW, "tile of %d atoms exceeds shared memory", s->tile_cap);
        launch_forces_fp64(a, s->g, s->pt, s->tile_cap, half(s), with_energy, s->stream);
    }
    CKL();
    if (ev.second) {
        CK(cudaEventRecord(ev.second, s->stream));
        s->ev_force.push_back(ev);
    }
    s->launches += force_kernels(s);
    s->force_evals += 1;
    s->forces_valid = true;
    return MD_OK;
}

int ensure_lists(md_system* s) {
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state: call md_set_state first");
    if (!s->lists_valid) return do_build(s);
    return MD_OK;
}

// LJ constants of every species pair (FP64 and the mixed path's FP32 copies); returns the
// largest cutoff.  rcut may be NULL (r_cut for every pair).
double fill_pair_table(PairTable& pt, const double* eps, const double* sigma, const double* rcut, double r_cut) {
    double rcmax = 0.0;
    for (int t = 0; t < pt.nsp * pt.nsp; ++t) {
        const double e = eps[t], sg = sigma[t];
        const double rc_t = rcut ? rcut[t] : r_cut;
        rcmax = std::max(rcmax, rc_t);
        pt.sig_d[t] = sg;
        pt.sig2_d[t] = sg * sg;
        pt.eps_d[t] = e;
        pt.rc2_d[t] = rc_t * rc_t;
        pt.sig2_f[t] = (float)(sg * sg);
        pt.c48_f[t] = (float)(48.0 * e * 2048.0);
        pt.c24_f[t] = (float)(24.0 * e * 2048.0);
        pt.c4_f[t] = (float)(4.0 * e);
        pt.rc2_f[t] = (float)(rc_t * rc_t);
    }
    return rcmax;
}

// The mixed kernels' FP64 decision band around r_cut^2, from the cell width, the skin and
// the smallest pair cutoff (tile_frame_cut_band).
void set_cut_band(md_system* s) {
    double rc2_min = s->pt.rc2_d[0];
    for (int t = 1; t < s->pt.nsp * s->pt.nsp; ++t) rc2_min = std::min(rc2_min, s->pt.rc2_d[t]);
    const double wmax = std::max(s->g.w[0], std::max(s->g.w[1], s->g.w[2]));
    s->pt.cut_band = (float)tile_frame_cut_band(wmax, 0.5 * s->skin, std::sqrt(rc2_min));
    set_band_thresholds(s->pt);
}

int validate_params(md_system* s, const md_params* p, double r_cut) {
    if (!p) return fail(s, MD_ERR_ARG, "params is NULL");
    if (p->n_species < 1 || p->n_species > MAX_SPECIES)
        return fail(s, MD_ERR_ARG, "n_species must be in [1, %d]", MAX_SPECIES);
    if (!p->eps || !p->sigma || !p->mass) return fail(s, MD_ERR_ARG, "eps, sigma and mass are required");
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(s, MD_ERR_ARG, "dt must be positive");
    if (p->precision != MD_FP64 && p->precision != MD_MIXED) return fail(s, MD_ERR_ARG, "bad precision");
    if (p->list_kind != MD_LIST_FULL && p->list_kind != MD_LIST_HALF_COLOUR8 &&
        p->list_kind != MD_LIST_HALF_ATOMIC_FREE)
        return fail(s, MD_ERR_ARG, "bad list kind");
    if (p->list_kind == MD_LIST_HALF_ATOMIC_FREE && p->precision != MD_MIXED)
        return fail(s, MD_ERR_ARG, "MD_LIST_HALF_ATOMIC_FREE needs MD_MIXED");
    if (p->rebuild != MD_REBUILD_SKIN_HALF && p->rebuild != MD_REBUILD_EVERY_K)
        return fail(s, MD_ERR_ARG, "bad rebuild policy");
    if (p->rebuild == MD_REBUILD_EVERY_K && p->rebuild_k < 1) return fail(s, MD_ERR_ARG, "rebuild_k must be >= 1");
    const int ns = p->n_species;
    for (int a = 0; a < ns; ++a) {
        if (!(p->mass[a] > 0.0)) return fail(s, MD_ERR_ARG, "mass must be positive");
        for (int b = 0; b < ns; ++b) {
            const double e = p->eps[a * ns + b], sg = p->sigma[a * ns + b];
            const double rc = p->rcut ? p->rcut[a * ns + b] : r_cut;
            if (!(e >= 0.0) || !(sg > 0.0) || !(rc > 0.0) || !std::isfinite(e) || !std::isfinite(sg) ||
                !std::isfinite(rc))
                return fail(s, MD_ERR_ARG, "bad LJ parameters for pair (%d,%d)", a, b);
            if (e != p->eps[b * ns + a] || sg != p->sigma[b * ns + a] ||
                (p->rcut && rc != p->rcut[b * ns + a]))
                return fail(s, MD_ERR_ARG, "pair tables must be symmetric");
        }
    }
    return MD_OK;
}

// ---- graph-captured time steps
//
// One step = integrate -> step control (sets the IF condition) -> IF(rebuild){binning,
// gather, copy back, list build} -> forces.  Kernel arguments are fixed at capture,
// which is why the state always lives in st[0].  Captured for the first step of a call
// (half kick + drift) and for the following ones (closing + opening kick + drift).
void destroy_graph(md_system::StepGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = md_system::StepGraph{};
}

int capture_step(md_system* s, int mode, md_system::StepGraph& out) {
    destroy_graph(out);
    cudaStream_t cs = s->cap_stream;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    out.graph = g;
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const DevState& a = s->st[0];
    launch_integrate(a, s->g, s->pt, mode, mixed(s), s->dt, s->lim2, cs);
    launch_step_ctrl(s->rebuild == MD_REBUILD_EVERY_K ? 1 : 0, s->rebuild_k, a.rebuild_flag, s->d_ctrl,
                     s->d_ctrl + 1, a.err, h, cs);
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));  // all reserved bytes must be zero
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (s->timing) {
        auto ev = take_events(s);
        s->ev_free.push_back(ev);
        CK(cudaEventRecordWithFlags(ev.first, cs, cudaEventRecordExternal));
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        out.ev_a = ndeps ? deps[0] : nullptr;
        enqueue_forces(s, 0, cs);
        CK(cudaEventRecordWithFlags(ev.second, cs, cudaEventRecordExternal));
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        out.ev_b = ndeps ? deps[0] : nullptr;
    } else {
        enqueue_forces(s, 0, cs);
    }
    CK(cudaStreamEndCapture(cs, &g));
    // the rebuild body
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_bin(s, a, cs);
    cudaMemsetAsync(a.stats, 0, 4 * sizeof(int32_t), cs);
    enqueue_lists(s, a, cs);
    launch_count_build(s->d_ctrl + 1, cs);
    CK(cudaStreamEndCapture(cs, &body));
    CKL();
    CK(cudaGraphInstantiate(&out.exec, g, 0));
    return MD_OK;
}

// Fused step (full-list mixed path): step control -> IF(rebuild){binning, gather, list
// build, all on coordinate buffer p} -> force kernel with the velocity-Verlet epilogue
// (kkd: closing + opening kick and drift into buffer 1-p; else the closing kick only).
int capture_fused(md_system* s, bool kkd, int p, md_system::StepGraph& out) {
    destroy_graph(out);
    cudaStream_t cs = s->cap_stream;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    out.graph = g;
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const DevState a = view(s, p);
    launch_step_ctrl(s->rebuild == MD_REBUILD_EVERY_K ? 1 : 0, s->rebuild_k, a.rebuild_flag, s->d_ctrl,
                     s->d_ctrl + 1, a.err, h, cs);
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));  // all reserved bytes must be zero
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    const int mode = kkd ? FUSE_KICK_KICK_DRIFT : FUSE_KICK;
    if (s->timing) {
        auto ev = take_events(s);
        s->ev_free.push_back(ev);
        CK(cudaEventRecordWithFlags(ev.first, cs, cudaEventRecordExternal));
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        out.ev_a = ndeps ? deps[0] : nullptr;
        launch_forces_mixed_fused(a, s->g, s->pt, s->to, s->tile_cap, mode, step_out(s, 1 - p), s->dt, s->lim2, cs);
        CK(cudaEventRecordWithFlags(ev.second, cs, cudaEventRecordExternal));
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        out.ev_b = ndeps ? deps[0] : nullptr;
    } else {
        launch_forces_mixed_fused(a, s->g, s->pt, s->to, s->tile_cap, mode, step_out(s, 1 - p), s->dt, s->lim2, cs);
    }
    CK(cudaStreamEndCapture(cs, &g));
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_bin(s, a, cs);
    cudaMemsetAsync(a.stats, 0, 4 * sizeof(int32_t), cs);
    launch_build_lists(a, s->g, s->to, s->rl2, s->list_cap, s->tile_cap, 0, cs);
    launch_count_build(s->d_ctrl + 1, cs);
    CK(cudaStreamEndCapture(cs, &body));
    CKL();
    CK(cudaGraphInstantiate(&out.exec, g, 0));
    return MD_OK;
}

// MULTI_STEPS fused kick-kick-drift steps in one graph: the sequence of capture_fused,
// step after step, each with its own conditional rebuild node and alternating buffers.
constexpr int MULTI_STEPS = 8;

int capture_fused_multi(md_system* s, md_system::StepGraph& out) {
    destroy_graph(out);
    cudaStream_t cs = s->cap_stream;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    out.graph = g;
    std::vector<cudaGraphNode_t> tail;
    for (int j = 0; j < MULTI_STEPS; ++j) {
        const int p = j & 1;
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        CK(cudaStreamBeginCaptureToGraph(cs, g, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(),
                                         cudaStreamCaptureModeThreadLocal));
        const DevState a = view(s, p);
        launch_step_ctrl(s->rebuild == MD_REBUILD_EVERY_K ? 1 : 0, s->rebuild_k, a.rebuild_flag, s->d_ctrl,
                         s->d_ctrl + 1, a.err, h, cs);
        cudaStreamCaptureStatus status;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
        std::memset(cp_raw, 0, sizeof(cp_raw));  // all reserved bytes must be zero
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        CK(cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        CK(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        // under timing, event nodes around the first step's force kernel (each launch points
        // them at fresh events): one launch in MULTI_STEPS is timed, so that the events
        // barely change the steps they measure
        const bool timed = s->timing && j == 0;
        if (timed) {
            auto ev = take_events(s);
            s->ev_free.push_back(ev);
            CK(cudaEventRecordWithFlags(ev.first, cs, cudaEventRecordExternal));
            CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
            out.ev_multi_a.push_back(ndeps ? deps[0] : nullptr);
        }
        launch_forces_mixed_fused(a, s->g, s->pt, s->to, s->tile_cap, FUSE_KICK_KICK_DRIFT, step_out(s, 1 - p), s->dt,
                                  s->lim2, cs);
        if (timed) {
            auto ev = take_events(s);
            s->ev_free.push_back(ev);
            CK(cudaEventRecordWithFlags(ev.second, cs, cudaEventRecordExternal));
            CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
            out.ev_multi_b.push_back(ndeps ? deps[0] : nullptr);
        }
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps));
        tail.assign(deps, deps + ndeps);
        CK(cudaStreamEndCapture(cs, &g));
        CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        enqueue_bin(s, a, cs);
        cudaMemsetAsync(a.stats, 0, 4 * sizeof(int32_t), cs);
        launch_build_lists(a, s->g, s->to, s->rl2, s->list_cap, s->tile_cap, 0, cs);
        launch_count_build(s->d_ctrl + 1, cs);
        CK(cudaStreamEndCapture(cs, &body));
    }
    CKL();
    CK(cudaGraphInstantiate(&out.exec, g, 0));
    return MD_OK;
}

int ensure_graphs(md_system* s) {
    if (s->graphs_valid && s->graph_tile_cap == s->tile_cap && s->graph_list_cap == s->list_cap &&
        s->graph_timing == s->timing)
        return MD_OK;
    int rc;
    if (fused(s)) {
        for (int k = 0; k < 2; ++k)
            for (int p = 0; p < 2; ++p)
                if ((rc = capture_fused(s, k == 1, p, s->g_fused[k][p]))) return rc;
        if ((rc = capture_fused_multi(s, s->g_multi))) return rc;
    } else {
        if ((rc = capture_step(s, INT_KICK_DRIFT, s->g_first))) return rc;
        if ((rc = capture_step(s, INT_KICK_KICK_DRIFT, s->g_mid))) return rc;
    }
    s->graphs_valid = true;
    s->graph_tile_cap = s->tile_cap;
    s->graph_list_cap = s->list_cap;
    s->graph_timing = s->timing;
    return MD_OK;
}

// The same step sequence launched from the host, reading the rebuild flag after every
// step (for profilers, which do not see kernels inside conditional graph nodes).
int run_steps_direct(md_system* s, int len, bool first) {
    int rc;
    const DevState& a = s->st[0];
    for (int k = 0; k < len; ++k) {
        CK(cudaMemsetAsync(a.rebuild_flag, 0, sizeof(int32_t), s->stream));
        launch_integrate(a, s->g, s->pt, (first && k == 0) ? INT_KICK_DRIFT : INT_KICK_KICK_DRIFT, mixed(s), s->dt,
                         s->lim2, s->stream);
        CKL();
        s->launches += 1;
        if ((rc = sync_flags(s))) return rc;
        const long long step = s->n_steps + k + 1;
        bool rebuild = s->h_flags[1] != 0;
        if (s->rebuild == MD_REBUILD_EVERY_K) {
            const bool due = (step % s->rebuild_k) == 0;
            if (rebuild && !due) return fail(s, MD_ERR_SKIN_VIOLATION, "an atom moved more than skin/2");
            rebuild = due;
        }
        if (rebuild && (rc = do_build(s))) return rc;
        if ((rc = do_forces(s, 0))) return rc;
    }
    return MD_OK;
}

// The fused step sequence launched from the host (see run_chunk_fused).
int run_steps_direct_fused(md_system* s, int len, bool first, bool last) {
    int rc;
    const DevState a = view(s, 0);
    if (first) {
        CK(cudaMemsetAsync(a.rebuild_flag, 0, sizeof(int32_t), s->stream));
        launch_integrate(a, s->g, s->pt, INT_KICK_DRIFT, 1, s->dt, s->lim2, s->stream);
        CKL();
        s->launches += 1;
    }
    int p = 0;
    for (int k = 0; k < len; ++k) {
        if ((rc = sync_flags(s))) return rc;
        const long long step = s->n_steps + k + 1;
        bool rebuild = s->h_flags[1] != 0;
        if (s->rebuild == MD_REBUILD_EVERY_K) {
            const bool due = (step % s->rebuild_k) == 0;
            if (rebuild && !due) return fail(s, MD_ERR_SKIN_VIOLATION, "an atom moved more than skin/2");
            rebuild = due;
        }
        CK(cudaMemsetAsync(a.rebuild_flag, 0, sizeof(int32_t), s->stream));
        if (rebuild && (rc = do_build(s, p))) return rc;
        const bool kkd = !(last && k == len - 1);
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (s->timing) {
            ev = take_events(s);
            CK(cudaEventRecord(ev.first, s->stream));
        }
        launch_forces_mixed_fused(view(s, p), s->g, s->pt, s->to, s->tile_cap,
                                  kkd ? FUSE_KICK_KICK_DRIFT : FUSE_KICK, step_out(s, 1 - p), s->dt, s->lim2,
                                  s->stream);
        CKL();
        if (ev.second) {
            CK(cudaEventRecord(ev.second, s->stream));
            s->ev_force.push_back(ev);
        }
        s->launches += 1;
        s->force_evals += 1;
        if (kkd) p ^= 1;
    }
    if (p && (rc = positions_to_buffer0(s))) return rc;
    s->forces_valid = last;
    return MD_OK;
}

// A chunk of len fused steps.  Step j's force kernel also performs the closing kick of
// step j and, unless it is the last step of the md_step call, the opening kick and drift
// of step j+1; the first step of a call starts with a plain kick + drift.  Coordinates
// alternate between the two FP32 buffers and end the chunk in buffer 0.
int run_chunk_fused(md_system* s, int len, bool first, bool last) {
    int rc;
    if (!s->use_graphs) return run_steps_direct_fused(s, len, first, last);
    if ((rc = ensure_graphs(s))) return rc;
    const DevState a = view(s, 0);
    launch_copy_state(s->st[2], a, s->stream);
    CKL();
    s->launches += 1;
    s->snapshot_first = first;
    s->h_ctrl[0] = s->n_steps;
    s->h_ctrl[1] = 0;
    CK(cudaMemcpyAsync(s->d_ctrl, s->h_ctrl, 2 * sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    if (first) {
        // the displacement flag of a later chunk's first step comes from the previous one
        CK(cudaMemsetAsync(a.rebuild_flag, 0, sizeof(int32_t), s->stream));
        launch_integrate(a, s->g, s->pt, INT_KICK_DRIFT, 1, s->dt, s->lim2, s->stream);
        CKL();
        s->launches += 1;
    }
    int p = 0;
    const int n_kkd = last ? len - 1 : len;  // steps that end with the next opening kick and drift
    for (int k = 0; k < len; ++k) {
        if (s->g_multi.exec && p == 0 && k + MULTI_STEPS <= n_kkd) {
            if (s->timing) {
                const auto& gm = s->g_multi;
                for (size_t j = 0; j < gm.ev_multi_a.size() && j < gm.ev_multi_b.size(); ++j) {
                    if (!gm.ev_multi_a[j] || !gm.ev_multi_b[j]) continue;
                    auto ev = take_events(s);
                    CK(cudaGraphExecEventRecordNodeSetEvent(gm.exec, gm.ev_multi_a[j], ev.first));
                    CK(cudaGraphExecEventRecordNodeSetEvent(gm.exec, gm.ev_multi_b[j], ev.second));
                    s->ev_force.push_back(ev);
                }
            }
            CK(cudaGraphLaunch(s->g_multi.exec, s->stream));  // MULTI_STEPS steps; back in buffer 0
            s->launches += 2 * MULTI_STEPS;
            s->force_evals += MULTI_STEPS;
            k += MULTI_STEPS - 1;
            continue;
        }
        const bool kkd = !(last && k == len - 1);
        md_system::StepGraph& gr = s->g_fused[kkd ? 1 : 0][p];
        if (s->timing && gr.ev_a && gr.ev_b) {
            auto ev = take_events(s);
            CK(cudaGraphExecEventRecordNodeSetEvent(gr.exec, gr.ev_a, ev.first));
            CK(cudaGraphExecEventRecordNodeSetEvent(gr.exec, gr.ev_b, ev.second));
            s->ev_force.push_back(ev);
        }
        CK(cudaGraphLaunch(gr.exec, s->stream));
        s->launches += 2;  // step control, fused force kernel
        s->force_evals += 1;
        if (kkd) p ^= 1;
    }
    if (p && (rc = positions_to_buffer0(s))) return rc;
    CK(cudaMemcpyAsync(s->h_ctrl, s->d_ctrl, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    if ((rc = sync_flags(s))) return rc;
    const uint32_t e = s->h_flags[0];
    if (e & ERR_TILE_OVERFLOW) return MD_ERR_CELL_OVERFLOW;  // the chunk is redone: nothing of it counts
    if (e & ERR_LIST_OVERFLOW) return MD_ERR_LIST_OVERFLOW;
    const long long builds = s->h_ctrl[1];
    s->launches += builds * 10;  // binning (8), list build, build counter
    if (builds > 0) {
        s->n_builds += builds;
        s->max_list = (int)s->h_flags[2];
        s->max_tile = (int)s->h_flags[3];
        s->list_entries = (int64_t)((uint64_t)s->h_flags[4] | ((uint64_t)s->h_flags[5] << 32));
    }
    s->forces_valid = last;
    return check_err(s, ERR_NONFINITE | ERR_ESCAPE | ERR_SKIN);
}

// Run len graph-launched steps; read the device status once at the end.
int run_chunk(md_system* s, int len, bool first) {
    int rc;
    if (!s->use_graphs) return run_steps_direct(s, len, first);
    if ((rc = ensure_graphs(s))) return rc;
    const DevState& a = s->st[0];
    // snapshot of the chunk's starting state (for a redo after a capacity overflow)
    launch_copy_state(s->st[2], a, s->stream);
    CKL();
    s->launches += 1;
    s->snapshot_first = first;
    s->h_ctrl[0] = s->n_steps;
    s->h_ctrl[1] = 0;
    CK(cudaMemcpyAsync(s->d_ctrl, s->h_ctrl, 2 * sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemsetAsync(a.rebuild_flag, 0, sizeof(int32_t), s->stream));
    for (int k = 0; k < len; ++k) {
        md_system::StepGraph& gr = (first && k == 0) ? s->g_first : s->g_mid;
        if (s->timing && gr.ev_a && gr.ev_b) {
            auto ev = take_events(s);
            CK(cudaGraphExecEventRecordNodeSetEvent(gr.exec, gr.ev_a, ev.first));
            CK(cudaGraphExecEventRecordNodeSetEvent(gr.exec, gr.ev_b, ev.second));
            s->ev_force.push_back(ev);
        }
        CK(cudaGraphLaunch(gr.exec, s->stream));
        s->launches += 2 + force_kernels(s);  // integrate, step control, forces
        s->force_evals += 1;
    }
    CK(cudaMemcpyAsync(s->h_ctrl, s->d_ctrl, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    if ((rc = sync_flags(s))) return rc;
    const uint32_t e = s->h_flags[0];
    if (e & ERR_TILE_OVERFLOW) return MD_ERR_CELL_OVERFLOW;  // the chunk is redone: nothing of it counts
    if (e & ERR_LIST_OVERFLOW) return MD_ERR_LIST_OVERFLOW;
    const long long builds = s->h_ctrl[1];
    s->launches += builds * 10;  // binning (8), list build, build counter
    if (builds > 0) {
        s->n_builds += builds;
        s->max_list = (int)s->h_flags[2];
        s->max_tile = (int)s->h_flags[3];
        s->list_entries = (int64_t)((uint64_t)s->h_flags[4] | ((uint64_t)s->h_flags[5] << 32));
    }
    return check_err(s, ERR_NONFINITE | ERR_ESCAPE | ERR_SKIN);
}

// Capacities for the rebuilds inside the next chunk of graph-launched steps: a chunk that
// outgrows them is redone from its snapshot, so grow them ahead of need once the last
// build came close to a limit (lists are kept; the graphs are captured again).
int ensure_headroom(md_system* s) {
    if (s->max_list + std::max(16, s->max_list / 4) > s->list_cap) {
        const int cap = list_cap_for(s->max_list);
        if (cap <= 65535) {
            int rc = alloc_lists(s, cap, true);
            if (rc) return rc;
        }
    }
    if (s->max_tile + std::max(64, s->max_tile / 8) > s->tile_cap) {
        const int cap = std::min(round_up(s->max_tile + s->max_tile / 4 + 64, 32), round_up((int)s->n + 1, 32));
        if (cap > s->tile_cap && cap <= 32767 && list_smem(s, s->list_cap, cap) <= 226 * 1024 &&
            fsmem(s, 0, cap) <= 226 * 1024)
            s->tile_cap = cap;
    }
    return MD_OK;
}

int restore_snapshot(md_system* s) {
    // back to the chunk's starting state; rebuild with capacity regrowth; forces again
    const int saved_list = s->max_list, saved_tile = s->max_tile;
    launch_copy_state(s->st[0], s->st[2], s->stream);
    CKL();
    CK(cudaMemsetAsync(s->st[0].err, 0, sizeof(uint32_t), s->stream));
    // grow what overflowed (the device counters hold the sizes the failed build needed)
    int rc = sync_flags(s);
    if (rc) return rc;
    const int need_list = std::max((int)s->h_flags[2], saved_list);
    const int need_tile = std::max((int)s->h_flags[3], saved_tile);
    if (need_list > s->list_cap && (rc = alloc_lists(s, std::min(list_cap_for(need_list), 65535)))) return rc;
    if (need_tile > s->tile_cap) {
        // the rebuild in the chunk needed larger tiles than the restored state has: keep
        // the grown capacity through the rebuild below (which otherwise fits it to the
        // restored state), or the redone chunk would overflow again
        s->tile_cap = std::min(round_up(need_tile + need_tile / 4 + 64, 32), round_up((int)s->n + 1, 32));
        s->tile_cap = std::max(s->tile_cap, need_tile);
        s->tile_floor = std::max(s->tile_floor, s->tile_cap);
    }
    s->lists_valid = false;
    s->forces_valid = false;
    if ((rc = do_build(s))) return rc;
    CK(cudaMemsetAsync(s->st[0].rebuild_flag, 0, sizeof(int32_t), s->stream));
    return do_forces(s, 0);
}

}  // namespace

extern "C" {

int md_create(int64_t n, const double box[3], double r_cut, double skin, const md_params* p, md_system** out) {
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    md_system* s = new md_system();
    auto bail = [&](int code) {
        md_destroy(s);
        return code;
    };
    if (n < 0 || n > 0x7fffffffLL - 64) return bail(MD_ERR_ARG);
    if (!box || !(r_cut > 0.0) || !(skin >= 0.0) || !std::isfinite(r_cut) || !std::isfinite(skin))
        return bail(MD_ERR_ARG);
    int rc = validate_params(s, p, r_cut);
    if (rc) return bail(rc);
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(p->stream);
    init_force_kernels();
    init_list_kernels();
    init_grad_kernels();
    init_tbsma_kernels();
    init_half_af_kernels();
    {
        const char* ng = std::getenv("MDGB_NO_GRAPHS");
        s->use_graphs = !(ng && ng[0] && ng[0] != '0');
        const char* nf = std::getenv("MDGB_NO_FUSE");
        s->no_fuse = nf && nf[0] && nf[0] != '0';
        const char* nc = std::getenv("MDGB_NO_COMPACT");
        s->no_compact = nc && nc[0] && nc[0] != '0';
        const char* fg = std::getenv("MDGB_FIT_GRID");
        s->fit_grid = fg && fg[0] && fg[0] != '0';
    }
    s->n = n;
    s->np = round_up((int)std::max<int64_t>(n, 1), 64);
    s->precision = p->precision;
    s->list_kind = p->list_kind;
    s->rebuild = p->rebuild;
    s->rebuild_k = p->rebuild_k;
    s->dt = p->dt;
    s->skin = skin;
    // pair table and the list radius
    const int ns = p->n_species;
    PairTable& pt = s->pt;
    pt.nsp = ns;
    const double rcmax = fill_pair_table(pt, p->eps, p->sigma, p->rcut, r_cut);
    for (int a = 0; a < ns; ++a) {
        pt.mass[a] = p->mass[a];
        pt.hdtm[a] = (0.5 * p->dt) / p->mass[a];
        pt.hdtm_q[a] = pt.hdtm[a] * 0x1p-32;
    }
    s->rcut = rcmax;
    s->rcut_default = r_cut;
    s->rl = rcmax + skin;
    s->rl2 = s->rl * s->rl;
    const double half_skin = 0.5 * skin;
    s->lim2 = half_skin * half_skin;
    // cell grid: per dimension the largest multiple of 4 cells at least r_list wide (8
    // colour classes of 2x2x2 blocks); full lists, which need no colours, take 6 where
    // that would leave 4 (a tile that is the whole box)
    Geometry& g = s->g;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) return bail(MD_ERR_ARG);
        s->box[d] = box[d];
        const int fit = (int)std::min(std::floor(box[d] / (s->rl * (1.0 + 1e-12))), 1024.0);
        const int nc = grid_cells(fit, s->list_kind == MD_LIST_FULL);
        if (nc < 4) {
            fail(s, MD_ERR_BOX_TOO_SMALL, "box side %g < 4 r_list", box[d]);
            return bail(MD_ERR_BOX_TOO_SMALL);
        }
        g.L[d] = box[d];
        g.nc[d] = nc;
        g.w[d] = box[d] / nc;
        g.inv_w[d] = nc / box[d];
        for (int t = 0; t < 4; ++t) s->to.off[d][t] = (float)((t - 1.5) * g.w[d]);
    }
    set_block_layout(g);
    set_cut_band(s);
    // initial capacities from the mean density (regrown on overflow)
    const double vol = box[0] * box[1] * box[2];
    const double rho = (double)n / vol;
    const double tile_vol = 64.0 * g.w[0] * g.w[1] * g.w[2];
    s->tile_cap = round_up((int)std::ceil(rho * tile_vol * 1.5) + 64, 64);
    s->tile_cap = std::min(s->tile_cap, round_up((int)n + 1, 32));
    const double sphere = 4.0 / 3.0 * M_PI * s->rl * s->rl * s->rl * rho;
    // half lists are about half as long on average, but the first atom of a cell lists
    // every later atom of its cell as well, so both kinds start from the full estimate
    int lc = (int)std::ceil(sphere * 1.4) + 16;
    lc = round_up(std::min(lc, 512), 8);

    // workspace
    for (int k = 0; k < 3; ++k) {
        DevState& d = s->st[k];
        d.n = n;
        d.np = s->np;
        if ((rc = dalloc(s, &d.x, n)) || (rc = dalloc(s, &d.y, n)) || (rc = dalloc(s, &d.z, n)) ||
            (rc = dalloc(s, &d.vx, n)) || (rc = dalloc(s, &d.vy, n)) || (rc = dalloc(s, &d.vz, n)) ||
            (rc = dalloc(s, &d.ix, n)) || (rc = dalloc(s, &d.iy, n)) || (rc = dalloc(s, &d.iz, n)) ||
            (rc = dalloc(s, &d.species, n)) || (rc = dalloc(s, &d.orig, n)))
            return bail(rc);
    }
    DevState& d0 = s->st[0];
    if ((rc = dalloc(s, &d0.rx, n)) || (rc = dalloc(s, &d0.ry, n)) || (rc = dalloc(s, &d0.rz, n)) ||
        (rc = dalloc(s, &d0.cell_of, n)) || (rc = dalloc(s, &d0.xr, n)) || (rc = dalloc(s, &d0.xr_ref, n)))
        return bail(rc);
    if ((rc = dalloc(s, &d0.cell_start, (size_t)g.ncell + 1)) || (rc = dalloc(s, &d0.centre, 3 * (size_t)g.ncell)) ||
        (rc = dalloc(s, &d0.nl_cnt, n)) ||
        (rc = dalloc(s, &d0.err, 1)) || (rc = dalloc(s, &d0.rebuild_flag, 1)) || (rc = dalloc(s, &d0.stats, 8)) ||
        (rc = dalloc(s, &d0.blk_list, (size_t)g.nblock)) ||
        (p->list_kind == MD_LIST_HALF_ATOMIC_FREE && (rc = dalloc(s, &d0.af_steps, (size_t)g.nblock * 8 * 14 * 2))))
        return bail(rc);
    if (p->precision == MD_MIXED) {
        if ((rc = dalloc(s, &d0.fq, 3 * (size_t)n)) || (rc = dalloc(s, &d0.pe_atom_f, n)) ||
            (rc = dalloc(s, &d0.vir_atom_f, 6 * (size_t)n)) || (rc = dalloc(s, &s->xr_alt, n)) ||
            (rc = dalloc(s, &s->pos_alt, 3 * (size_t)n)))
            return bail(rc);
    } else {
        if ((rc = dalloc(s, &d0.f, 3 * (size_t)n)) || (rc = dalloc(s, &d0.pe_atom_d, n)) ||
            (rc = dalloc(s, &d0.vir_atom_d, 6 * (size_t)n)))
            return bail(rc);
    }
    d0.ncell = g.ncell;
    s->ncell_alloc = g.ncell;
    if (upload_centres(s) != MD_OK) return bail(MD_ERR_CUDA);
    for (int k = 1; k < 3; ++k) {
        DevState& d1 = s->st[k];
        d1.cell_start = d0.cell_start;
        d1.centre = d0.centre;
        d1.ncell = d0.ncell;
        d1.nl_cnt = d0.nl_cnt;
        d1.err = d0.err;
        d1.rebuild_flag = d0.rebuild_flag;
        d1.stats = d0.stats;
        d1.blk_list = d0.blk_list;
        d1.af_steps = d0.af_steps;
        d1.fq = d0.fq;
        d1.f = d0.f;
        d1.pe_atom_f = d0.pe_atom_f;
        d1.vir_atom_f = d0.vir_atom_f;
        d1.pe_atom_d = d0.pe_atom_d;
        d1.vir_atom_d = d0.vir_atom_d;
    }
    if ((rc = dalloc(s, &s->d_ctrl, 2))) return bail(rc);
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MD_ERR_CUDA);
    if ((rc = alloc_lists(s, lc))) return bail(rc);
    if ((rc = dalloc(s, &s->atom_cell, n)) || (rc = dalloc(s, &s->cell_count, g.ncell)) ||
        (rc = dalloc(s, &s->cursor, g.ncell)) || (rc = dalloc(s, &s->slot_key, n)) ||
        (rc = dalloc(s, &s->slot_src, n)) || (rc = dalloc(s, &s->sorted_src, n)) ||
        (rc = dalloc(s, &s->scan_scratch, scan_scratch_ints(g.ncell))))
        return bail(rc);
    s->nparts = 592;
    if ((rc = dalloc(s, &s->partials, 8 * (size_t)s->nparts)) || (rc = dalloc(s, &s->out8, 8))) return bail(rc);
    if (cudaMallocHost(&s->h_flags, 16 * sizeof(uint32_t)) != cudaSuccess) return bail(MD_ERR_CUDA);
    if (cudaMallocHost(&s->h_ctrl, 2 * sizeof(long long)) != cudaSuccess) return bail(MD_ERR_CUDA);
    if (cudaMemsetAsync(d0.err, 0, sizeof(uint32_t), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->d_ctrl, 0, 2 * sizeof(long long), s->stream) != cudaSuccess ||
        cudaMemsetAsync(d0.rebuild_flag, 0, sizeof(int32_t), s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return bail(MD_ERR_CUDA);
    *out = s;
    return MD_OK;
}

int md_set_state(md_system* s, const double* pos, const double* vel, const int32_t* species, int device_ptrs) {
    if (!s) return MD_ERR_ARG;
    if (!pos) return fail(s, MD_ERR_ARG, "pos is NULL");
    DeviceGuard dg(s->device);
    const size_t n = (size_t)s->n;
    const double *dpos = pos, *dvel = vel;
    const int32_t* dsp = species;
    double* tmp = nullptr;
    int32_t* tsp = nullptr;
    if (!device_ptrs && n > 0) {
        CK(cudaMallocAsync(&tmp, sizeof(double) * 6 * n, s->stream));
        CK(cudaMemcpyAsync(tmp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
        dpos = tmp;
        if (vel) {
            CK(cudaMemcpyAsync(tmp + 3 * n, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
            dvel = tmp + 3 * n;
        }
        if (species) {
            CK(cudaMallocAsync(&tsp, sizeof(int32_t) * n, s->stream));
            CK(cudaMemcpyAsync(tsp, species, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream));
            dsp = tsp;
        }
    }
    s->cur = 0;
    CK(cudaMemsetAsync(s->st[0].err, 0, sizeof(uint32_t), s->stream));
    launch_set_state(s->st[0], dpos, dvel, dsp, s->pt.nsp, s->stream);
    CKL();
    if (tmp) CK(cudaFreeAsync(tmp, s->stream));
    if (tsp) CK(cudaFreeAsync(tsp, s->stream));
    int rc = sync_flags(s);
    if (rc) return rc;
    s->has_state = false;
    s->lists_valid = false;
    s->forces_valid = false;
    if (s->h_flags[0] & 0x80000000u) return fail(s, MD_ERR_ARG, "species id out of range");
    if (s->h_flags[0] & 0x40000000u) return fail(s, MD_ERR_NONFINITE, "non-finite position or velocity");
    s->has_state = true;
    return MD_OK;
}

int md_bin_cells(md_system* s) {
    if (!s) return MD_ERR_ARG;
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    DeviceGuard dg(s->device);
    CK(cudaMemsetAsync(s->st[0].err, 0, sizeof(uint32_t), s->stream));
    int rc = do_bin(s);
    if (rc) return rc;
    rc = sync_flags(s);
    if (rc) return rc;
    return check_err(s, ~0u);
}

int md_build_neighbors(md_system* s) {
    if (!s) return MD_ERR_ARG;
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    DeviceGuard dg(s->device);
    return do_build(s);
}

int md_forces(md_system* s, double* f_out, int device_ptrs) {
    if (!s) return MD_ERR_ARG;
    DeviceGuard dg(s->device);
    int rc = ensure_lists(s);
    if (rc) return rc;
    rc = do_forces(s, 0);
    if (rc) return rc;
    if (f_out && s->n > 0) {
        const size_t n = (size_t)s->n;
        if (device_ptrs) {
            launch_forces_out(s->st[s->cur], mixed(s), f_out, s->stream);
            CKL();
        } else {
            double* tmp = nullptr;
            CK(cudaMallocAsync(&tmp, sizeof(double) * 3 * n, s->stream));
            launch_forces_out(s->st[s->cur], mixed(s), tmp, s->stream);
            CKL();
            CK(cudaMemcpyAsync(f_out, tmp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaFreeAsync(tmp, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        }
    }
    rc = sync_flags(s);
    if (rc) return rc;
    return check_err(s, ERR_NONFINITE | ERR_TILE_OVERFLOW);
}

int md_step(md_system* s, int32_t n_steps) {
    if (!s) return MD_ERR_ARG;
    if (n_steps < 0) return fail(s, MD_ERR_ARG, "n_steps < 0");
    if (n_steps == 0 || s->n == 0) {
        s->n_steps += n_steps;
        return MD_OK;
    }
    DeviceGuard dg(s->device);
    int rc = ensure_lists(s);
    if (rc) return rc;
    if (!s->forces_valid && (rc = do_forces(s, 0))) return rc;
    // chunks of graph-launched steps; the host reads the device status once per chunk
    constexpr int CHUNK = 200;
    int done = 0;
    int redo = 0;
    while (done < n_steps) {
        const int len = std::min(CHUNK, n_steps - done);
        const bool first = done == 0;
        if ((rc = ensure_headroom(s))) return rc;
        rc = fused(s) ? run_chunk_fused(s, len, first, done + len == n_steps) : run_chunk(s, len, first);
        if (rc == MD_ERR_CELL_OVERFLOW || rc == MD_ERR_LIST_OVERFLOW) {
            // a rebuild inside the chunk outgrew the captured capacities: restore the
            // chunk's starting state, rebuild with regrowth on the host, and redo it
            if (++redo > 4) return rc;
            s->n_redos++;
            if ((rc = restore_snapshot(s))) return rc;
            continue;
        }
        if (rc) return rc;
        done += len;
        s->n_steps += len;
        redo = 0;
    }
    if (!fused(s)) {
        // the closing half kick of the last step (fused steps apply it in the force kernel)
        launch_integrate(s->st[0], s->g, s->pt, INT_KICK, mixed(s), s->dt, s->lim2, s->stream);
        CKL();
        s->launches += 1;
    }
    rc = sync_flags(s);
    if (rc) return rc;
    return check_err(s, ERR_NONFINITE | ERR_ESCAPE | ERR_SKIN);
}

int md_set_params(md_system* s, const double* eps, const double* sigma, const double* rcut) {
    if (!s) return MD_ERR_ARG;
    if (!eps || !sigma) return fail(s, MD_ERR_ARG, "eps and sigma are required");
    const int ns = s->pt.nsp;
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b) {
            const int t = a * ns + b, u = b * ns + a;
            const double rc = rcut ? rcut[t] : s->rcut_default;
            if (!(eps[t] >= 0.0) || !(sigma[t] > 0.0) || !(rc > 0.0) || !std::isfinite(eps[t]) ||
                !std::isfinite(sigma[t]) || !std::isfinite(rc))
                return fail(s, MD_ERR_ARG, "bad LJ parameters for pair (%d,%d)", a, b);
            if (eps[t] != eps[u] || sigma[t] != sigma[u] || (rcut && rcut[t] != rcut[u]))
                return fail(s, MD_ERR_ARG, "pair tables must be symmetric");
            if (rc > s->rcut) return fail(s, MD_ERR_ARG, "cutoff %g exceeds the %g the lists were sized for", rc, s->rcut);
        }
    DeviceGuard dg(s->device);
    // kernels read the table by value: queued work keeps the old one, captured graphs are redone
    fill_pair_table(s->pt, eps, sigma, rcut, s->rcut_default);
    set_cut_band(s);
    s->potential = 0;
    s->forces_valid = false;
    s->graphs_valid = false;
    return MD_OK;
}

int md_colour_conflicts(md_system* s, int32_t n_phases, int64_t* conflicts) {
    if (!s || !conflicts || (n_phases != 1 && n_phases != 8)) return MD_ERR_ARG;
    if (n_phases == 8 && s->g.linear) return fail(s, MD_ERR_ARG, "linear block numbering has no colour classes");
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    DeviceGuard dg(s->device);
    *conflicts = 0;
    if (s->n == 0) return MD_OK;
    int rc = ensure_lists(s);  // a current binning
    if (rc) return rc;
    int32_t* tags = nullptr;
    unsigned long long* cnt = nullptr;
    CK(cudaMallocAsync(&tags, sizeof(int32_t) * (size_t)s->n, s->stream));
    CK(cudaMallocAsync(&cnt, sizeof(unsigned long long), s->stream));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s->stream));
    const int per = s->g.nblock / n_phases;
    for (int c = 0; c < n_phases; ++c) {
        CK(cudaMemsetAsync(tags, 0xff, sizeof(int32_t) * (size_t)s->n, s->stream));  // -1: unclaimed
        launch_colour_tags(s->st[0], s->g, c * per, per, tags, cnt, s->stream);
        CKL();
    }
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(tags, s->stream));
    CK(cudaFreeAsync(cnt, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    *conflicts = (int64_t)h;
    return MD_OK;
}

int md_set_tbsma(md_system* s, double A, double xi, double p, double q, double r0, double r_cut) {
    if (!s) return MD_ERR_ARG;
    const double v[6] = {A, xi, p, q, r0, r_cut};
    for (double x : v)
        if (!std::isfinite(x) || !(x > 0.0)) return fail(s, MD_ERR_ARG, "TB-SMA parameters must be positive");
    if (!mixed(s) || half(s) || s->pt.nsp != 1)
        return fail(s, MD_ERR_ARG, "TB-SMA needs one species, MD_MIXED and MD_LIST_FULL");
    if (r_cut > s->rcut) return fail(s, MD_ERR_ARG, "cutoff %g exceeds the %g the lists were sized for", r_cut, s->rcut);
    // the density terms go through the fixed-point split: psi(0) = xi^2 exp(2q) must stay below 2048
    if (!(xi * xi * std::exp(2.0 * q) < 2000.0)) return fail(s, MD_ERR_ARG, "xi^2 exp(2q) must be below 2000");
    DeviceGuard dg(s->device);
    if (!s->emb) {
        int rc = dalloc(s, &s->emb, (size_t)std::max<int64_t>(s->n, 1));
        if (rc) return rc;
    }
    const double ln2 = std::log(2.0);
    TBTable& tb = s->tb;
    tb.r0 = (float)r0;
    tb.kp = (float)(-p / (r0 * ln2));
    tb.lp = (float)std::log2(A);
    tb.kq = (float)(-2.0 * q / (r0 * ln2));
    tb.lq = (float)(2.0 * std::log2(xi));
    tb.c_rep = (float)(2.0 * p / r0);
    tb.c_band = (float)(q / r0);
    tb.rc2_d = r_cut * r_cut;
    const double wmax = std::max(s->g.w[0], std::max(s->g.w[1], s->g.w[2]));
    const double band = tile_frame_cut_band(wmax, 0.5 * s->skin, r_cut);
    tb.rc2lo_f = (float)(r_cut * r_cut * (1.0 - band));
    tb.rc2hi_f = (float)(r_cut * r_cut * (1.0 + band));
    s->potential = 1;
    s->forces_valid = false;
    s->graphs_valid = false;
    return MD_OK;
}

// dL/dx, dL/deps, dL/dsigma for dL/dF = grad_f, and/or dE/deps, dE/dsigma
static int backward(md_system* s, const double* grad_f, int device_ptrs, double* grad_pos, double* grad_eps,
                    double* grad_sigma, double* de_deps, double* de_dsig) {
    if (!s) return MD_ERR_ARG;
    DeviceGuard dg(s->device);
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state: call md_set_state first");
    if (half(s)) return fail(s, MD_ERR_ARG, "derivatives need full neighbour lists (MD_LIST_FULL)");
    if (s->potential != 0) return fail(s, MD_ERR_ARG, "derivatives are for the Lennard-Jones potential");
    const int ns = s->pt.nsp;
    const int ncol = ns * ns * 4;
    std::vector<double> tot(ncol, 0.0);
    if (s->n > 0) {
        int rc = ensure_lists(s);
        if (rc) return rc;
        const int64_t n = s->n;
        const int nparts = 256;
        double* scratch = nullptr;
        double *G = nullptr, *gx = nullptr;
        CK(cudaMallocAsync(&scratch, sizeof(double) * backward_scratch_doubles(n, ns, nparts), s->stream));
        if (grad_f) {
            if (device_ptrs) {
                G = const_cast<double*>(grad_f);
            } else {
                CK(cudaMallocAsync(&G, sizeof(double) * 3 * n, s->stream));
                CK(cudaMemcpyAsync(G, grad_f, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
            }
        }
        if (grad_pos) {
            if (device_ptrs) gx = grad_pos;
            else CK(cudaMallocAsync(&gx, sizeof(double) * 3 * n, s->stream));
        }
        const size_t smem = backward_smem_bytes(!mixed(s), s->tile_cap);
        if (smem > 226 * 1024) return fail(s, MD_ERR_CELL_OVERFLOW, "tile of %d atoms exceeds shared memory", s->tile_cap);
        launch_force_backward(s->st[0], s->g, s->pt, s->to, s->tile_cap, !mixed(s), G, gx, de_deps != nullptr, scratch,
                              nparts, s->stream);
        CKL();
        s->launches += (G ? 1 : 0) + 1 + (gx ? 1 : 0) + 2;
        const double* totals = scratch + backward_scratch_doubles(n, ns, nparts) - ncol;
        CK(cudaMemcpyAsync(tot.data(), totals, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s->stream));
        if (grad_pos && !device_ptrs)
            CK(cudaMemcpyAsync(grad_pos, gx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
        if (grad_f && !device_ptrs) CK(cudaFreeAsync(G, s->stream));
        if (grad_pos && !device_ptrs) CK(cudaFreeAsync(gx, s->stream));
        CK(cudaFreeAsync(scratch, s->stream));
        if ((rc = sync_flags(s))) return rc;
        if ((rc = check_err(s, ERR_NONFINITE | ERR_TILE_OVERFLOW))) return rc;
    }
    // column (s_i * ns + s_j) * 4 + q holds the terms of atoms of species s_i with neighbours
    // of species s_j (each pair halved per side): the shared value of {a,b} gets both sides
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b) {
            const double* ab = &tot[(a * ns + b) * 4];
            const double* ba = &tot[(b * ns + a) * 4];
            const int t = a * ns + b;
            const double w = (a == b) ? 1.0 : 0.0;  // the diagonal entry already holds both sides
            if (grad_eps) grad_eps[t] = ab[0] + (1.0 - w) * ba[0];
            if (grad_sigma) grad_sigma[t] = ab[1] + (1.0 - w) * ba[1];
            if (de_deps) de_deps[t] = ab[2] + (1.0 - w) * ba[2];
            if (de_dsig) de_dsig[t] = ab[3] + (1.0 - w) * ba[3];
        }
    return MD_OK;
}

int md_forces_backward(md_system* s, const double* grad_f, int device_ptrs, double* grad_pos, double* grad_eps,
                       double* grad_sigma) {
    if (!s || !grad_f) return MD_ERR_ARG;
    return backward(s, grad_f, device_ptrs, grad_pos, grad_eps, grad_sigma, nullptr, nullptr);
}

int md_energy_param_grad(md_system* s, double* de_deps, double* de_dsigma) {
    if (!s || !de_deps || !de_dsigma) return MD_ERR_ARG;
    return backward(s, nullptr, 0, nullptr, nullptr, nullptr, de_deps, de_dsigma);
}

int md_energy_virial(md_system* s, double* pe, double* ke, double virial[6]) {
    if (!s) return MD_ERR_ARG;
    DeviceGuard dg(s->device);
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (s->n > 0) {
        int rc = ensure_lists(s);
        if (rc) return rc;
        if ((rc = do_forces(s, 1))) return rc;
        launch_reduce_energy(s->st[s->cur], s->pt, mixed(s), s->partials, s->nparts, s->out8, s->stream);
        CKL();
        s->launches += 2;
        CK(cudaMemcpyAsync(h, s->out8, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
        if ((rc = sync_flags(s))) return rc;
        if ((rc = check_err(s, ERR_NONFINITE | ERR_TILE_OVERFLOW))) return rc;
    }
    if (pe) *pe = h[0];
    if (ke) *ke = h[1];
    if (virial)
        for (int c = 0; c < 6; ++c) virial[c] = h[2 + c];
    return MD_OK;
}

int md_get_state(md_system* s, double* pos, double* vel, int32_t* image, int device_ptrs) {
    if (!s) return MD_ERR_ARG;
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    DeviceGuard dg(s->device);
    const size_t n = (size_t)s->n;
    if (n == 0) return MD_OK;
    if (device_ptrs) {
        launch_get_state(s->st[s->cur], pos, vel, image, s->stream);
        CKL();
        return MD_OK;
    }
    double* tmp = nullptr;
    int32_t* timg = nullptr;
    CK(cudaMallocAsync(&tmp, sizeof(double) * 6 * n, s->stream));
    CK(cudaMallocAsync(&timg, sizeof(int32_t) * 3 * n, s->stream));
    launch_get_state(s->st[s->cur], tmp, tmp + 3 * n, timg, s->stream);
    CKL();
    if (pos) CK(cudaMemcpyAsync(pos, tmp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    if (vel) CK(cudaMemcpyAsync(vel, tmp + 3 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    if (image) CK(cudaMemcpyAsync(image, timg, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(tmp, s->stream));
    CK(cudaFreeAsync(timg, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MD_OK;
}

int md_get_neighbors(md_system* s, int64_t* n_pairs, int32_t* pairs) {
    if (!s || !n_pairs) return MD_ERR_ARG;
    DeviceGuard dg(s->device);
    int rc = ensure_lists(s);
    if (rc) return rc;
    const int64_t npairs = half(s) ? s->list_entries : s->list_entries / 2;
    *n_pairs = npairs;
    if (!pairs || npairs == 0) return MD_OK;
    unsigned long long* counter = nullptr;
    int32_t* dp = nullptr;
    CK(cudaMallocAsync(&counter, sizeof(unsigned long long), s->stream));
    CK(cudaMallocAsync(&dp, sizeof(int32_t) * 2 * (size_t)npairs, s->stream));
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s->stream));
    launch_pairs_out(s->st[s->cur], s->g, half(s), counter, dp, npairs, s->stream);
    CKL();
    unsigned long long got = 0;
    CK(cudaMemcpyAsync(&got, counter, sizeof(got), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(pairs, dp, sizeof(int32_t) * 2 * (size_t)npairs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(counter, s->stream));
    CK(cudaFreeAsync(dp, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if ((int64_t)got != npairs) return fail(s, MD_ERR_STATE, "pair count mismatch (%llu vs %lld)", got, (long long)npairs);
    std::vector<int64_t> keys((size_t)npairs);
    for (int64_t k = 0; k < npairs; ++k) keys[k] = ((int64_t)pairs[2 * k] << 32) | (uint32_t)pairs[2 * k + 1];
    std::sort(keys.begin(), keys.end());
    for (int64_t k = 0; k < npairs; ++k) {
        pairs[2 * k] = (int32_t)(keys[k] >> 32);
        pairs[2 * k + 1] = (int32_t)(keys[k] & 0xffffffff);
    }
    return MD_OK;
}

int md_get_cells(md_system* s, int32_t* cell_of_atom) {
    if (!s || !cell_of_atom) return MD_ERR_ARG;
    if (!s->has_state) return fail(s, MD_ERR_STATE, "no state");
    DeviceGuard dg(s->device);
    if (s->n == 0) return MD_OK;
    int32_t* tmp = nullptr;
    CK(cudaMallocAsync(&tmp, sizeof(int32_t) * (size_t)s->n, s->stream));
    launch_cells_out(s->st[s->cur], s->g, tmp, s->stream);
    CKL();
    CK(cudaMemcpyAsync(cell_of_atom, tmp, sizeof(int32_t) * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(tmp, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MD_OK;
}

int md_get_info(md_system* s, md_info* out) {
    if (!s || !out) return MD_ERR_ARG;
    out->n = s->n;
    for (int d = 0; d < 3; ++d) {
        out->ncell[d] = s->g.nc[d];
        out->cell_width[d] = s->g.w[d];
    }
    out->list_cap = s->list_cap;
    out->tile_cap = s->tile_cap;
    out->n_builds = s->n_builds;
    out->n_steps = s->n_steps;
    out->list_entries = s->list_entries;
    out->max_list = s->max_list;
    out->max_tile = s->max_tile;
    out->kernel_launches = s->launches;
    out->force_evals = s->force_evals;
    out->force_ms = s->force_ms;
    out->timed_force_evals = s->timed_force;
    out->build_ms = s->build_ms;
    out->timed_builds = s->timed_build;
    out->n_redos = s->n_redos;
    return MD_OK;
}

int md_set_timing(md_system* s, int enable) {
    if (!s) return MD_ERR_ARG;
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    drain_events(s);
    s->timing = enable != 0;
    s->force_ms = s->build_ms = 0.0;
    s->timed_force = s->timed_build = 0;
    return MD_OK;
}

int md_last_error(md_system* s, char* buf, int64_t len) {
    if (!s || !buf || len <= 0) return MD_ERR_ARG;
    std::snprintf(buf, (size_t)len, "%s", s->msg);
    return MD_OK;
}

void md_destroy(md_system* s) {
    if (!s) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    for (void* p : s->allocs) cudaFree(p);
    s->allocs.clear();
    drain_events(s);
    for (auto& e : s->ev_free) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
    destroy_graph(s->g_first);
    destroy_graph(s->g_mid);
    for (auto& row : s->g_fused)
        for (auto& gr : row) destroy_graph(gr);
    destroy_graph(s->g_multi);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
