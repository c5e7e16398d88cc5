// oct_hydro.cu -- host side of the C ABI declared in include/oct_hydro.h:
// handle, validation, work list, launches, the RK3 CUDA graph and the
// autotuner.  The kernels live in rhs_kernel.cuh and step_kernels.cuh.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/oct_hydro.h"
#include "oct_common.cuh"
#include "rhs_launch.h"
#include "step_kernels.cuh"
#include "gravity.cuh"

namespace {
// An NVTX range around each ABI call that launches work, so that timelines
// (nsys, ncu --nvtx) show which call a kernel belongs to.  Without a tool
// attached NVTX calls cost a pointer test.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

using namespace octh;

static thread_local std::string g_last_error;

static oct_status fail(oct_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

// For the other translation units of the library (diagnostics).
oct_status octh_fail_text(oct_status st, const char *msg) { return fail(st, "%s", msg); }

#define CUDA_TRY(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? OCT_E_NOMEM : OCT_E_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                     \
    } while (0)

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
};

struct oct_hydro {
    int device = 0, n_sm = 0;
    int n_sub = 0, edge0 = 0, n_species = 0, nf = 0;
    double gamma = 5.0 / 3.0;
    int precision = OCT_FP64;
    double cfl = 0.4, rho_floor = 1e-12, eps1 = 1e-3, eps2 = 0.1, dt_cap = 0.0;
    int bc = OCT_BC_GIVEN;
    bool layout_ok = false;
    // host copies
    std::vector<int> edge;
    std::vector<long long> off, doff;
    std::vector<double> dx;
    std::vector<int> nbr;
    std::vector<WorkItem> items;
    std::vector<int> item_begin;
    std::vector<int> order;             // execution order of the items (empty: index order)
    int items_mode = -1, items_grid = 0;  // the launch shape the items were cut for
    long long state_len = 0, rhs_len = 0;
    // launch shape: 0 8x8 tiles (6x6 for edge 12), 256 threads; 1 8x4 tiles (6x4
    // for edge 12), 256 threads; 2 8x8 tiles, 512 threads; 3 8x8 tiles, 1024 threads
    int tile_mode = 0;
    // [form][tile mode], form = precision + 2 * recon
    int ctas_per_sm[4][RHS_MODES] = {};  // the occupancy limit (0: the shape does not fit)
    int combine_ctas[2] = {1, 1};  // resident combine CTAs per SM: [0] stages 2/3, [1] stage 1
    int cta_use[4][RHS_MODES] = {};      // resident CTAs per SM of the persistent grid (0: the limit)
    int recon = OCT_RECON_CONSERVED;
    double *d_Wprim = nullptr;   // primitive variables of the state (primitive reconstruction)
    // device memory
    int *d_edge = nullptr, *d_nbr = nullptr, *d_item_begin = nullptr;
    // per subgrid, set by the whole-subgrid uniform test before each RHS: the
    // ghosted block held one value per field ([0..n) the step's state, as of
    // the first stage; [n..2n) the stage state of stages 2 and 3)
    int *d_sub_uniform = nullptr;
    // per subgrid, by the same test (FP64): the fields whose ghosted block
    // held one value, for the subgrids the RHS kernel then took
    unsigned *d_field_uni = nullptr;
    int *d_changed = nullptr;  // per subgrid: interior changed by the last combine (stages 2 and 3)
    bool uni_test = false;     // the last RHS launch ran the uniform test
    // record of the stage state W written by the combines of stages 1 and 2:
    // per subgrid one value per field (uniform pass) and that value
    int *d_out_uni = nullptr;
    double *d_out_val = nullptr;
    // record of the interiors of the state a step starts from (first stage)
    int *d_u_uni = nullptr;
    double *d_u_val = nullptr;
    // the RHS launch's work list after the uniform test (live_items_kernel)
    WorkItem *d_live_items = nullptr;
    int *d_live_slot = nullptr, *d_n_live = nullptr;
    bool items_live_split = false;
    bool ghosts_sourced = false;  // uniform level on which every ghost cell has a source
    long long *d_off = nullptr, *d_doff = nullptr;
    double *d_dx = nullptr;
    WorkItem *d_items = nullptr;
    int *d_order = nullptr;   // execution order (null: index order)
    int *d_ticket = nullptr;  // dynamic-scheduling counters of the RHS kernel (zero between launches)
    double *d_dtcap = nullptr;  // dt cap of oct_hydro_rk_step (0: none), read by the captured graph
    double *d_dt_part = nullptr;  // per-block minima of dt_blocks_kernel
    int *d_dt_count = nullptr;    // its blocks-done counter (zero between launches)
    double *d_amax_tile = nullptr, *d_dt = nullptr, *d_W = nullptr, *d_L = nullptr, *d_Uhost = nullptr,
           *d_Lhost = nullptr;
    unsigned *d_flags = nullptr;
    int2 *d_amr_plan = nullptr;  // ghost-cell sources across levels (OCT_BC_AMR)
    std::vector<int32_t> amr_level, amr_origin;  // the levels as last set, for a rebuild
    int amr_root = 0, amr_periodic = 0;
    int prolong_order = 0;  // 0 injection, 1 limited linear
    bool has_prolong = false;  // the plan holds limited linear prolongations
    double *d_faces = nullptr;     // boundary face fluxes of the subgrids next to a level change
    int *d_face_slot = nullptr;    // per subgrid: its slot in d_faces, or -1
    RefluxCorr *d_corr = nullptr;  // flux corrections at coarse-fine faces, grouped by coarse cell
    int *d_corr_first = nullptr;
    int n_corr_cells = 0;
    std::map<const double *, GraphEntry> graphs;
    // same-level monopole gravity: the stencil for the radius last used
    int *d_gst_off = nullptr;
    GravEntry *d_gst_k = nullptr;
    int gst_n = 0, gst_S = 0;
    double gst_rs = 0.0;
};

template <class P>
static void dfree(P *&p)
{
    if (p)
        cudaFree((void *)p);
    p = nullptr;
}

// Makes the handle's device current for the duration of an ABI call and
// restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(const oct_hydro *h)
    {
        int cur = -1;
        if (h && cudaGetDevice(&cur) == cudaSuccess && cur != h->device && cudaSetDevice(h->device) == cudaSuccess)
            prev = cur;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

static void drop_graphs(oct_hydro *h)
{
    for (auto &kv : h->graphs)
        if (kv.second.exec)
            cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

static void free_layout(oct_hydro *h)
{
    dfree(h->d_edge);
    dfree(h->d_nbr);
    dfree(h->d_item_begin);
    dfree(h->d_sub_uniform);
    dfree(h->d_field_uni);
    dfree(h->d_changed);
    dfree(h->d_out_uni);
    dfree(h->d_out_val);
    dfree(h->d_u_uni);
    dfree(h->d_u_val);
    dfree(h->d_live_items);
    dfree(h->d_live_slot);
    dfree(h->d_n_live);
    dfree(h->d_off);
    dfree(h->d_doff);
    dfree(h->d_dx);
    dfree(h->d_items);
    dfree(h->d_order);
    dfree(h->d_amax_tile);
    dfree(h->d_W);
    dfree(h->d_L);
    dfree(h->d_Uhost);
    dfree(h->d_Lhost);
    dfree(h->d_amr_plan);
    dfree(h->d_faces);
    dfree(h->d_face_slot);
    dfree(h->d_corr);
    dfree(h->d_corr_first);
    dfree(h->d_Wprim);
    h->n_corr_cells = 0;
    drop_graphs(h);
}

static oct_status set_kernel_attrs(oct_hydro *h)
{
    for (int form = 0; form < 4; form++)
        for (int mode = 0; mode < RHS_MODES; mode++) {
            int nb = 0;
            CUDA_TRY(rhs_prepare(form, mode, h->nf, &nb));
            h->ctas_per_sm[form][mode] = nb;
        }
    // the default 8x8 / 256-thread shape must fit
    for (int form = 0; form < 4; form++)
        if (h->ctas_per_sm[form][0] < 1)
            return fail(OCT_E_CUDA, "RHS kernel does not fit on an SM (%zu bytes shared memory)",
                        rhs_smem_bytes(h->nf, form, 0));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->combine_ctas[0], combine_kernel<false>,
                                                           COMBINE_THREADS, 0));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->combine_ctas[1], combine_kernel<true>,
                                                           COMBINE_THREADS, 0));
    h->combine_ctas[0] = std::max(h->combine_ctas[0], 1);
    h->combine_ctas[1] = std::max(h->combine_ctas[1], 1);
    return OCT_OK;
}

static int form_of(const oct_hydro *h) { return h->precision + 2 * h->recon; }

// CTAs of the persistent RHS grid for the current form and launch shape.
static int grid_ctas(const oct_hydro *h)
{
    const int form = form_of(h), mode = h->tile_mode;
    const int per_sm = h->cta_use[form][mode] > 0 ? h->cta_use[form][mode] : h->ctas_per_sm[form][mode];
    return h->n_sm * std::max(per_sm, 1);
}

// Work items for the current launch shape.  Each subgrid is cut into tiles of
// the shape's capacity (6 wide for edge 12).  When the tiles are all of one
// size and do not fill the last round of the persistent grid -- r = N mod G
// items left over for G CTAs, r at most G/2 -- the last r tiles are cut in
// half along y: the last round then runs 2r half tiles (each a little over
// half the work of a tile: the ring of halo cells grows) instead of r whole
// tiles while G - r CTAs wait.  With mixed sizes the execution order is by
// estimated work, largest first, and the kernel hands out items dynamically.
// A subgrid's items stay contiguous (item_begin).
static void build_items(oct_hydro *h)
{
    const int G = grid_ctas(h);
    h->items.clear();
    h->order.clear();
    h->item_begin.assign(h->n_sub + 1, 0);
    bool same = true;
    long long n_tiles = 0;
    for (int s = 0; s < h->n_sub; s++) {
        const int E = h->edge[s];
        const int tx = (E == 12) ? 6 : 8, ty = (h->tile_mode == 1) ? 4 : tx;
        n_tiles += (long long)(E / tx) * (E / ty);
        same = same && E == h->edge[0];
    }
    const int ty0 = (h->tile_mode == 1) ? 4 : (h->edge[0] == 12 ? 6 : 8);
    const long long r = n_tiles % G;
    const long long split_from = (same && r > 0 && 2 * r <= G && ty0 % 2 == 0) ? n_tiles - r : n_tiles;
    // the work list after the uniform test may cut its own last round in
    // half when the static items are all whole tiles of an even height >= 4
    h->items_live_split = same && split_from == n_tiles && ty0 % 2 == 0 && ty0 >= 4;
    long long k = 0;
    for (int s = 0; s < h->n_sub; s++) {
        h->item_begin[s] = (int)h->items.size();
        const int E = h->edge[s];
        const int tx = (E == 12) ? 6 : 8;
        const int ty = (h->tile_mode == 1) ? 4 : tx;
        for (int y0 = 0; y0 < E; y0 += ty)
            for (int x0 = 0; x0 < E; x0 += tx, k++) {
                const int parts = k >= split_from ? 2 : 1;
                for (int p = 0; p < parts; p++) {
                    WorkItem w;
                    w.s = s;
                    w.x0 = x0;
                    w.y0 = y0 + p * (ty / parts);
                    w.txty = tx | ((ty / parts) << 8);
                    h->items.push_back(w);
                }
            }
    }
    h->item_begin[h->n_sub] = (int)h->items.size();
    if (!same) {
        // largest first: cells plus the halo ring, times the planes
        auto work = [&](const WorkItem &w) {
            const int tx = w.txty & 0xFF, ty = (w.txty >> 8) & 0xFF;
            return (long long)(tx * ty + tx + ty) * (h->edge[w.s] + 2);
        };
        h->order.resize(h->items.size());
        for (size_t i = 0; i < h->items.size(); i++)
            h->order[i] = (int)i;
        std::stable_sort(h->order.begin(), h->order.end(),
                         [&](int a, int b) { return work(h->items[a]) > work(h->items[b]); });
    }
    h->items_mode = h->tile_mode;
    h->items_grid = G;
}

static oct_status upload_items(oct_hydro *h)
{
    dfree(h->d_items);
    dfree(h->d_item_begin);
    dfree(h->d_amax_tile);
    dfree(h->d_order);
    dfree(h->d_sub_uniform);
    dfree(h->d_field_uni);
    dfree(h->d_changed);
    dfree(h->d_out_uni);
    dfree(h->d_out_val);
    dfree(h->d_u_uni);
    dfree(h->d_u_val);
    dfree(h->d_live_items);
    dfree(h->d_live_slot);
    dfree(h->d_n_live);
    CUDA_TRY(cudaMalloc(&h->d_sub_uniform, sizeof(int) * 2 * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_field_uni, sizeof(unsigned) * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_changed, sizeof(int) * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_out_uni, sizeof(int) * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMemset(h->d_out_uni, 0, sizeof(int) * std::max(1, h->n_sub)));  // W holds nothing known
    CUDA_TRY(cudaMalloc(&h->d_out_val, sizeof(double) * MAXNF * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_live_items, sizeof(WorkItem) * 2 * std::max<size_t>(1, h->items.size())));
    CUDA_TRY(cudaMalloc(&h->d_live_slot, sizeof(int) * 2 * std::max<size_t>(1, h->items.size())));
    CUDA_TRY(cudaMalloc(&h->d_n_live, sizeof(int)));
    CUDA_TRY(cudaMalloc(&h->d_u_uni, sizeof(int) * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_u_val, sizeof(double) * MAXNF * std::max(1, h->n_sub)));
    CUDA_TRY(cudaMalloc(&h->d_items, sizeof(WorkItem) * h->items.size()));
    CUDA_TRY(cudaMemcpy(h->d_items, h->items.data(), sizeof(WorkItem) * h->items.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->d_item_begin, sizeof(int) * h->item_begin.size()));
    CUDA_TRY(cudaMemcpy(h->d_item_begin, h->item_begin.data(), sizeof(int) * h->item_begin.size(),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->d_amax_tile, sizeof(double) * std::max<size_t>(1, h->items.size())));
    if (!h->order.empty()) {
        CUDA_TRY(cudaMalloc(&h->d_order, sizeof(int) * h->order.size()));
        CUDA_TRY(cudaMemcpy(h->d_order, h->order.data(), sizeof(int) * h->order.size(), cudaMemcpyHostToDevice));
    }
    return OCT_OK;
}

// Re-cuts the work items when the launch shape or the grid changed since they
// were built (precision, reconstruction or autotuning); captured step graphs
// hold the old items and are dropped.  Called before any RHS launch, outside
// graph capture.
static oct_status sync_items(oct_hydro *h)
{
    if (h->items_mode == h->tile_mode && h->items_grid == grid_ctas(h))
        return OCT_OK;
    build_items(h);
    drop_graphs(h);
    return upload_items(h);
}

static bool valid_edge(int E)
{
    return E == 8 || E == 12 || E == 16;
}

extern "C" oct_status oct_hydro_create(int n_subgrids, int edge, int ghost, int n_species, double gamma,
                                       oct_hydro_t *out)
{
    if (!out)
        return fail(OCT_E_ARG, "out is NULL");
    *out = nullptr;
    if (n_subgrids <= 0)
        return fail(OCT_E_ARG, "n_subgrids must be positive (got %d)", n_subgrids);
    if (edge != 0 && !valid_edge(edge))
        return fail(OCT_E_ARG, "edge must be 8, 12, 16 or 0 (got %d)", edge);
    if (ghost != NG)
        return fail(OCT_E_ARG, "ghost must be 3 (got %d)", ghost);
    if (n_species < 0 || n_species > MAXNF - 6)
        return fail(OCT_E_ARG, "n_species must be in 0..%d (got %d)", MAXNF - 6, n_species);
    if (!(gamma > 1.0) || !std::isfinite(gamma))
        return fail(OCT_E_ARG, "gamma must be > 1 (got %g)", gamma);
    oct_hydro *h = new (std::nothrow) oct_hydro;
    if (!h)
        return fail(OCT_E_NOMEM, "host allocation failed");
    h->n_sub = n_subgrids;
    h->edge0 = edge;
    h->n_species = n_species;
    h->nf = 6 + n_species;
    h->gamma = gamma;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(OCT_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    oct_status st = set_kernel_attrs(h);
    if (st == OCT_OK && cudaMalloc(&h->d_flags, sizeof(unsigned)) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc flags");
    if (st == OCT_OK && cudaMemset(h->d_flags, 0, sizeof(unsigned)) != cudaSuccess)
        st = fail(OCT_E_CUDA, "cudaMemset flags");
    if (st == OCT_OK && cudaMalloc(&h->d_dt, sizeof(double)) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc dt");
    if (st == OCT_OK && cudaMalloc(&h->d_dt_part, sizeof(double) * DT_MAX_BLOCKS) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc dt partial minima");
    if (st == OCT_OK && cudaMalloc(&h->d_dt_count, sizeof(int)) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc dt counter");
    if (st == OCT_OK && cudaMemset(h->d_dt_count, 0, sizeof(int)) != cudaSuccess)
        st = fail(OCT_E_CUDA, "cudaMemset dt counter");
    if (st == OCT_OK && cudaMalloc(&h->d_dtcap, sizeof(double)) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc dt cap");
    if (st == OCT_OK && cudaMemset(h->d_dtcap, 0, sizeof(double)) != cudaSuccess)
        st = fail(OCT_E_CUDA, "cudaMemset dt cap");
    if (st == OCT_OK && cudaMalloc(&h->d_ticket, 2 * sizeof(int)) != cudaSuccess)
        st = fail(OCT_E_NOMEM, "cudaMalloc ticket");
    if (st == OCT_OK && cudaMemset(h->d_ticket, 0, 2 * sizeof(int)) != cudaSuccess)
        st = fail(OCT_E_CUDA, "cudaMemset ticket");
    if (st != OCT_OK) {
        oct_hydro_destroy(h);
        return st;
    }
    if (edge != 0) {
        std::vector<double> dxv(n_subgrids, 1.0 / edge);
        st = oct_hydro_set_layout(h, nullptr, nullptr, dxv.data(), nullptr, nullptr, OCT_BC_GIVEN);
        if (st != OCT_OK) {
            std::string keep = g_last_error;
            oct_hydro_destroy(h);
            g_last_error = keep;
            return st;
        }
    }
    *out = h;
    return OCT_OK;
}

// Whether every ghost cell of a uniform level has a source: after the
// zero-gradient clamp along the axes without a face neighbour, the direction
// left (if any) has a neighbour.
static bool ghosts_all_sourced(const std::vector<int> &nb, int n)
{
    auto slot = [](int dx, int dy, int dz) {
        const int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
        return k > 13 ? k - 1 : k;
    };
    for (int t = 0; t < n; t++)
        for (int k = 0; k < 27; k++) {
            if (k == 13)
                continue;
            const int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
            int e[3] = {d[0], d[1], d[2]};
            for (int a = 0; a < 3; a++)
                if (d[a] != 0) {
                    int f[3] = {0, 0, 0};
                    f[a] = d[a];
                    if (nb[26 * (size_t)t + slot(f[0], f[1], f[2])] < 0)
                        e[a] = 0;
                }
            if ((e[0] | e[1] | e[2]) != 0 && nb[26 * (size_t)t + slot(e[0], e[1], e[2])] < 0)
                return false;
        }
    return true;
}

extern "C" oct_status oct_hydro_set_layout(oct_hydro_t h, const int32_t *edges, const int64_t *offsets,
                                           const double *dx, const int32_t *level, const int32_t *neighbours, int bc)
{
    DeviceGuard device_guard(h);
    (void)level;
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (bc < OCT_BC_GIVEN || bc > OCT_BC_OUTFLOW)
        return fail(OCT_E_ARG, "bc must be 0, 1 or 2 (got %d)", bc);
    const int n = h->n_sub;
    std::vector<int> edge(n);
    for (int s = 0; s < n; s++) {
        edge[s] = edges ? edges[s] : h->edge0;
        if (!valid_edge(edge[s]))
            return fail(OCT_E_ARG, "edge of subgrid %d must be 8, 12 or 16 (got %d)", s, edge[s]);
    }
    if (!dx && (h->dx.size() != (size_t)n))
        return fail(OCT_E_ARG, "dx is required");
    std::vector<double> dxv(n);
    for (int s = 0; s < n; s++) {
        dxv[s] = dx ? dx[s] : h->dx[s];
        if (!(dxv[s] > 0.0) || !std::isfinite(dxv[s]))
            return fail(OCT_E_ARG, "dx of subgrid %d must be positive (got %g)", s, dxv[s]);
    }
    const int nf = h->nf;
    std::vector<long long> off(n), doff(n);
    long long state_len = 0, rhs_len = 0;
    std::vector<std::pair<long long, long long>> spans(n);
    for (int s = 0; s < n; s++) {
        long long B = edge[s] + 2 * NG;
        long long len = nf * B * B * B;
        if (offsets) {
            off[s] = offsets[s];
            if (off[s] < 0 || off[s] % 4 != 0)
                return fail(OCT_E_ARG, "offset of subgrid %d must be a non-negative multiple of 4 doubles (got %lld)",
                            s, (long long)off[s]);
        } else {
            off[s] = state_len;
        }
        spans[s] = {off[s], off[s] + len};
        state_len = std::max(state_len, off[s] + len);
        if (!offsets)
            state_len = (state_len + 3) / 4 * 4;
        doff[s] = rhs_len;
        rhs_len += nf * (long long)edge[s] * edge[s] * edge[s];
    }
    std::sort(spans.begin(), spans.end());
    for (int s = 1; s < n; s++)
        if (spans[s].first < spans[s - 1].second)
            return fail(OCT_E_ARG, "subgrid blocks overlap in the state array");
    std::vector<int> nb;
    if (bc != OCT_BC_GIVEN) {
        if (!neighbours)
            return fail(OCT_E_ARG, "a neighbour table is required for periodic/outflow ghosts");
        for (int s = 1; s < n; s++)
            if (edge[s] != edge[0])
                return fail(OCT_E_ARG, "ghost exchange needs one common edge");
        nb.assign(neighbours, neighbours + 26 * (size_t)n);
        for (size_t i = 0; i < nb.size(); i++)
            if (nb[i] < -1 || nb[i] >= n)
                return fail(OCT_E_ARG, "neighbour entry %zu out of range (%d)", i, nb[i]);
    }
    const bool sourced = bc != OCT_BC_GIVEN && ghosts_all_sourced(nb, n);
    // commit
    free_layout(h);
    h->layout_ok = false;
    h->ghosts_sourced = sourced;
    h->edge = edge;
    h->dx = dxv;
    h->off = off;
    h->doff = doff;
    h->nbr = nb;
    h->bc = bc;
    h->state_len = state_len;
    h->rhs_len = rhs_len;
    build_items(h);
    CUDA_TRY(cudaMalloc(&h->d_edge, sizeof(int) * n));
    CUDA_TRY(cudaMemcpy(h->d_edge, edge.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->d_dx, sizeof(double) * n));
    CUDA_TRY(cudaMemcpy(h->d_dx, dxv.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->d_off, sizeof(long long) * n));
    CUDA_TRY(cudaMemcpy(h->d_off, off.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->d_doff, sizeof(long long) * n));
    CUDA_TRY(cudaMemcpy(h->d_doff, doff.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    if (!nb.empty()) {
        CUDA_TRY(cudaMalloc(&h->d_nbr, sizeof(int) * nb.size()));
        CUDA_TRY(cudaMemcpy(h->d_nbr, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice));
    }
    oct_status st = upload_items(h);
    if (st != OCT_OK)
        return st;
    if (h->recon == OCT_RECON_PRIMITIVE)
        CUDA_TRY(cudaMalloc(&h->d_Wprim, sizeof(double) * h->state_len));
    h->layout_ok = true;
    return OCT_OK;
}

extern "C" oct_status oct_hydro_set_reconstruction(oct_hydro_t h, int variables)
{
    DeviceGuard device_guard(h);
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (variables != OCT_RECON_CONSERVED && variables != OCT_RECON_PRIMITIVE)
        return fail(OCT_E_ARG, "variables must be OCT_RECON_CONSERVED or OCT_RECON_PRIMITIVE (got %d)", variables);
    if (variables == OCT_RECON_PRIMITIVE && h->layout_ok && !h->d_Wprim)
        CUDA_TRY(cudaMalloc(&h->d_Wprim, sizeof(double) * h->state_len));
    h->recon = variables;
    drop_graphs(h);
    return OCT_OK;
}

extern "C" oct_status oct_hydro_set_amr(oct_hydro_t h, const int32_t *level, const int32_t *origin, int root_cells,
                                        int periodic)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_set_amr");
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (!h->layout_ok)
        return fail(OCT_E_STATE, "no layout set");
    if (!level || !origin)
        return fail(OCT_E_ARG, "level and origin are required");
    const int n = h->n_sub, E = h->edge[0];
    for (int s = 0; s < n; s++)
        if (h->edge[s] != E)
            return fail(OCT_E_ARG, "ghost exchange needs one common edge");
    if (E % 2 != 0)
        return fail(OCT_E_ARG, "ghost exchange across levels needs an even edge (got %d)", E);
    if (root_cells <= 0 || root_cells % E != 0)
        return fail(OCT_E_ARG, "root_cells must be a positive multiple of the edge (got %d)", root_cells);
    // subgrid lookup by (level, subgrid coordinates)
    auto key = [](long long l, long long a, long long b, long long c) {
        return (((l * 4096 + a) * 4096 + b) * 4096) + c;
    };
    std::unordered_map<long long, int> at;
    for (int s = 0; s < n; s++) {
        const int l = level[s];
        if (l < 0 || l > 20)
            return fail(OCT_E_ARG, "level of subgrid %d out of range (%d)", s, l);
        const long long nl = (long long)root_cells << l;
        for (int a = 0; a < 3; a++)
            if (origin[3 * s + a] < 0 || origin[3 * s + a] % E != 0 || origin[3 * s + a] + E > nl)
                return fail(OCT_E_ARG, "origin of subgrid %d must be a multiple of %d inside its level", s, E);
        if (nl / E >= 4096)
            return fail(OCT_E_ARG, "too many subgrids per side at level %d", l);
        auto ins = at.emplace(key(l, origin[3 * s] / E, origin[3 * s + 1] / E, origin[3 * s + 2] / E), s);
        if (!ins.second)
            return fail(OCT_E_ARG, "subgrids %d and %d overlap", ins.first->second, s);
    }
    auto cover = [&](int l, const long long *c) -> int {
        if (l < 0)
            return -1;
        auto it = at.find(key(l, c[0] / E, c[1] / E, c[2] / E));
        return it == at.end() ? -1 : it->second;
    };
    const int B = E + 2 * NG;
    const int nzs = NG * B * B, nys = NG * B * E, nxs = NG * E * E;
    const int G = 2 * nzs + 2 * nys + 2 * nxs;
    std::vector<int2> plan((size_t)n * G);
    for (int s = 0; s < n; s++) {
        const int l = level[s];
        const long long nl = (long long)root_cells << l;
        for (int q = 0; q < G; q++) {
            int g[3];  // the enumeration of amr_ghost_kernel
            if (q < 2 * nzs) {
                const int r = q % nzs, side = q / nzs;
                g[0] = r % B - NG;
                g[1] = (r / B) % B - NG;
                g[2] = r / (B * B) + (side ? E : -NG);
            } else if (q < 2 * nzs + 2 * nys) {
                const int r0 = q - 2 * nzs, r = r0 % nys, side = r0 / nys;
                g[0] = r % B - NG;
                g[1] = (r / B) % NG + (side ? E : -NG);
                g[2] = r / (B * NG);
            } else {
                const int r0 = q - 2 * nzs - 2 * nys, r = r0 % nxs, side = r0 / nxs;
                g[0] = r % NG + (side ? E : -NG);
                g[1] = (r / NG) % E;
                g[2] = r / (NG * E);
            }
            long long c[3];
            for (int a = 0; a < 3; a++) {
                c[a] = (long long)origin[3 * s + a] + g[a];
                c[a] = periodic ? ((c[a] % nl) + nl) % nl : (c[a] < 0 ? 0 : (c[a] >= nl ? nl - 1 : c[a]));
            }
            auto local = [&](int t, const long long *p) {
                return ((p[2] - origin[3 * t + 2] + NG) * B + (p[1] - origin[3 * t + 1] + NG)) * B +
                       (p[0] - origin[3 * t] + NG);
            };
            int t = cover(l, c);
            if (t >= 0) {
                plan[(size_t)s * G + q] = make_int2(t, (int)local(t, c));
                continue;
            }
            const long long cc[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
            t = cover(l - 1, cc);
            if (t >= 0) {
                if (h->prolong_order == 0) {
                    plan[(size_t)s * G + q] = make_int2(t, (int)local(t, cc));  // injection: a copy
                } else {
                    // limited linear: bit 30; which half of the coarse cell per axis in
                    // bits 16..18 of y (the usable-slope mask follows below)
                    const int par = (int)((c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2));
                    plan[(size_t)s * G + q] = make_int2((int)(t | 0x40000000u), (int)local(t, cc) | (par << 16));
                }
                continue;
            }
            const long long cf[3] = {2 * c[0], 2 * c[1], 2 * c[2]};
            t = cover(l + 1, cf);
            if (t < 0)
                return fail(OCT_E_ARG, "ghost cell %d of subgrid %d has no source (levels not properly nested)", q, s);
            plan[(size_t)s * G + q] = make_int2((int)(t | 0x80000000u), (int)local(t, cf));
        }
    }
    // limited linear prolongation: a slope axis is usable when both coarse
    // neighbours are interior cells or ghosts filled by copy or restriction
    bool has_prolong = false;
    if (h->prolong_order == 1) {
        const long long B3 = (long long)B * B * B;
        std::vector<unsigned char> kind((size_t)n * B3, 0);  // 0 interior, 1 copy, 2 restriction, 3 prolongation
        for (int q = 0; q < G; q++) {
            int g[3];
            if (q < 2 * nzs) {
                const int r = q % nzs, side = q / nzs;
                g[0] = r % B - NG, g[1] = (r / B) % B - NG, g[2] = r / (B * B) + (side ? E : -NG);
            } else if (q < 2 * nzs + 2 * nys) {
                const int r0 = q - 2 * nzs, r = r0 % nys, side = r0 / nys;
                g[0] = r % B - NG, g[1] = (r / B) % NG + (side ? E : -NG), g[2] = r / (B * NG);
            } else {
                const int r0 = q - 2 * nzs - 2 * nys, r = r0 % nxs, side = r0 / nxs;
                g[0] = r % NG + (side ? E : -NG), g[1] = (r / NG) % E, g[2] = r / (NG * E);
            }
            const long long gl = ((long long)(g[2] + NG) * B + (g[1] + NG)) * B + (g[0] + NG);
            for (int s = 0; s < n; s++) {
                const int2 e = plan[(size_t)s * G + q];
                kind[(size_t)s * B3 + gl] = (e.x & 0x40000000) ? 3 : (e.x < 0 ? 2 : 1);
            }
        }
        const long long step[3] = {1, B, (long long)B * B};
        for (size_t i = 0; i < plan.size(); i++) {
            int2 &e = plan[i];
            if (!(e.x & 0x40000000) || e.x < 0)
                continue;
            has_prolong = true;
            const int t = e.x & 0x3FFFFFFF;
            const long long cl = e.y & 0xFFFF;
            int mask = 0;
            for (int a = 0; a < 3; a++)
                if (kind[(size_t)t * B3 + cl + step[a]] != 3 && kind[(size_t)t * B3 + cl - step[a]] != 3)
                    mask |= 1 << a;
            e.y |= mask << 19;
        }
    }
    // flux corrections: every face between a cell and a finer region
    struct Pending {
        long long cell;  // s * E^3 + interior linear index
        int s, k, side, t, u1, u2, t1, t2;
    };
    std::vector<Pending> pend;
    for (int s = 0; s < n; s++) {
        const int l = level[s];
        const long long nl = (long long)root_cells << l;
        for (int k = 0; k < 3; k++) {
            const int a1 = k == 0 ? 1 : 0, a2 = k == 2 ? 1 : 2;
            for (int side = 0; side < 2; side++)
                for (int t2 = 0; t2 < E; t2++)
                    for (int t1 = 0; t1 < E; t1++) {
                        int c[3];
                        c[k] = side ? E - 1 : 0;
                        c[a1] = t1;
                        c[a2] = t2;
                        long long g[3] = {(long long)origin[3 * s] + c[0], (long long)origin[3 * s + 1] + c[1],
                                          (long long)origin[3 * s + 2] + c[2]};
                        g[k] += side ? 1 : -1;
                        if (g[k] < 0 || g[k] >= nl) {
                            if (!periodic)
                                continue;
                            g[k] = ((g[k] % nl) + nl) % nl;
                        }
                        if (cover(l, g) >= 0)
                            continue;
                        long long fc[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
                        if (!side)
                            fc[k] += 1;
                        const int t = cover(l + 1, fc);
                        if (t < 0)
                            continue;
                        if (fc[k] - origin[3 * t + k] != (side ? 0 : E - 1))
                            return fail(OCT_E_ARG, "subgrids %d and %d overlap across levels", s, t);
                        pend.push_back({(long long)s * E * E * E + ((long long)c[2] * E + c[1]) * E + c[0], s, k, side,
                                        t, (int)(fc[a1] - origin[3 * t + a1]), (int)(fc[a2] - origin[3 * t + a2]), t1,
                                        t2});
                    }
        }
    }
    std::stable_sort(pend.begin(), pend.end(), [](const Pending &a, const Pending &b) { return a.cell < b.cell; });
    std::vector<int> slot(n, -1);
    int nslot = 0;
    for (const Pending &p : pend) {
        if (slot[p.s] < 0)
            slot[p.s] = nslot++;
        if (slot[p.t] < 0)
            slot[p.t] = nslot++;
    }
    const long long EE = (long long)E * E, fblk = 6LL * h->nf * EE;
    std::vector<RefluxCorr> corr;
    std::vector<int> first;
    for (size_t i = 0; i < pend.size(); i++) {
        const Pending &p = pend[i];
        if (i == 0 || p.cell != pend[i - 1].cell)
            first.push_back((int)corr.size());
        RefluxCorr C;
        C.d = h->doff[p.s] + (p.cell - (long long)p.s * E * E * E);
        C.fc = slot[p.s] * fblk + (2LL * p.k + p.side) * h->nf * EE + (long long)p.t2 * E + p.t1;
        C.ff = slot[p.t] * fblk + (2LL * p.k + (p.side ? 0 : 1)) * h->nf * EE + (long long)p.u2 * E + p.u1;
        C.s = p.s;
        C.side = p.side;
        corr.push_back(C);
    }
    first.push_back((int)corr.size());
    dfree(h->d_amr_plan);
    dfree(h->d_faces);
    dfree(h->d_face_slot);
    dfree(h->d_corr);
    dfree(h->d_corr_first);
    h->n_corr_cells = 0;
    CUDA_TRY(cudaMalloc(&h->d_amr_plan, sizeof(int2) * plan.size()));
    CUDA_TRY(cudaMemcpy(h->d_amr_plan, plan.data(), sizeof(int2) * plan.size(), cudaMemcpyHostToDevice));
    if (!corr.empty()) {
        CUDA_TRY(cudaMalloc(&h->d_faces, sizeof(double) * nslot * fblk));
        CUDA_TRY(cudaMalloc(&h->d_face_slot, sizeof(int) * n));
        CUDA_TRY(cudaMalloc(&h->d_corr, sizeof(RefluxCorr) * corr.size()));
        CUDA_TRY(cudaMalloc(&h->d_corr_first, sizeof(int) * first.size()));
        CUDA_TRY(cudaMemcpy(h->d_face_slot, slot.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->d_corr, corr.data(), sizeof(RefluxCorr) * corr.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->d_corr_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
        h->n_corr_cells = (int)first.size() - 1;
    }
    h->bc = OCT_BC_AMR;
    h->ghosts_sourced = false;
    h->has_prolong = has_prolong;
    h->amr_level.assign(level, level + n);
    h->amr_origin.assign(origin, origin + 3 * (size_t)n);
    h->amr_root = root_cells;
    h->amr_periodic = periodic;
    drop_graphs(h);
    return OCT_OK;
}

extern "C" oct_status oct_hydro_set_prolongation(oct_hydro_t h, int order)
{
    DeviceGuard device_guard(h);
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (order != 0 && order != 1)
        return fail(OCT_E_ARG, "prolongation order must be 0 (injection) or 1 (limited linear) (got %d)", order);
    const int prev = h->prolong_order;
    h->prolong_order = order;
    if (h->bc == OCT_BC_AMR && order != prev) {
        // rebuild the ghost plan with the new order from the levels as last set
        const std::vector<int32_t> lev = h->amr_level, org = h->amr_origin;
        const oct_status st = oct_hydro_set_amr(h, lev.data(), org.data(), h->amr_root, h->amr_periodic);
        if (st != OCT_OK) {
            h->prolong_order = prev;
            return st;
        }
    }
    return OCT_OK;
}

extern "C" oct_status oct_hydro_set_params(oct_hydro_t h, int precision, double cfl, double rho_floor,
                                           double de_switch1, double de_switch2)
{
    DeviceGuard device_guard(h);
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (precision != OCT_FP64 && precision != OCT_MIXED)
        return fail(OCT_E_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (!(cfl > 0.0 && cfl <= 1.0))
        return fail(OCT_E_ARG, "cfl must be in (0, 1] (got %g)", cfl);
    if (!(rho_floor >= 0.0) || !std::isfinite(rho_floor))
        return fail(OCT_E_ARG, "rho_floor must be >= 0");
    if (!(de_switch1 >= 0.0 && de_switch1 < 1.0) || !(de_switch2 >= 0.0 && de_switch2 < 1.0))
        return fail(OCT_E_ARG, "dual-energy switches must be in [0, 1)");
    h->precision = precision;
    h->cfl = cfl;
    h->rho_floor = rho_floor;
    h->eps1 = de_switch1;
    h->eps2 = de_switch2;
    drop_graphs(h);
    return OCT_OK;
}

extern "C" oct_status oct_hydro_set_dt_cap(oct_hydro_t h, double dt_cap)
{
    DeviceGuard device_guard(h);
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (std::isnan(dt_cap))
        return fail(OCT_E_ARG, "dt_cap is NaN");
    // the captured step graphs read the cap from device memory; wait for any
    // step in flight before changing it
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(h->d_dtcap, &dt_cap, sizeof(double), cudaMemcpyHostToDevice));
    h->dt_cap = dt_cap;
    return OCT_OK;
}

extern "C" int64_t oct_hydro_state_len(oct_hydro_t h)
{
    DeviceGuard device_guard(h);
    return h && h->layout_ok ? h->state_len : -1;
}

extern "C" int64_t oct_hydro_rhs_len(oct_hydro_t h)
{
    DeviceGuard device_guard(h);
    return h && h->layout_ok ? h->rhs_len : -1;
}

static oct_status check_ready(oct_hydro *h)
{
    if (!h)
        return fail(OCT_E_ARG, "handle is NULL");
    if (!h->layout_ok)
        return fail(OCT_E_STATE, "no layout set");
    return OCT_OK;
}

static oct_status check_ptr(const void *p, const char *name)
{
    if (!p)
        return fail(OCT_E_ARG, "%s is NULL", name);
    if ((uintptr_t)p % 16 != 0)
        return fail(OCT_E_ARG, "%s must be 16-byte aligned", name);
    return OCT_OK;
}

// Launches the RHS kernel of the handle's precision.
// Whether the stage states of a step can take the whole-subgrid uniform test
// from the combines' record (uniform level, every ghost sourced, the test on).
static bool record_test_ok(const oct_hydro *h)
{
    return (h->bc == OCT_BC_PERIODIC || h->bc == OCT_BC_OUTFLOW) && h->ghosts_sourced &&
           h->recon != OCT_RECON_PRIMITIVE;
}

// Whether an RHS launch takes its work list from live_items_kernel after the
// uniform test: one edge (no execution order), 8 or 16.
static bool live_ok(const oct_hydro *h)
{
    return h->recon != OCT_RECON_PRIMITIVE && !(h->bc == OCT_BC_AMR && h->n_corr_cells > 0) && h->order.empty() &&
           !h->edge.empty() && (h->edge[0] == 8 || h->edge[0] == 16);
}

// Whether the combines keep the record of W (uniform test on, record test
// possible).  W belongs to the handle and only the step writes it, so the
// record that stage 2 leaves describes W at the next step's start; a step
// without the record clears it (enqueue_step), as does a new layout.
static bool w_record_ok(const oct_hydro *h) { return h->uni_test && record_test_ok(h); }

// uni_slot: which half of the per-subgrid uniform flags the whole-subgrid
// test writes (1 for the stage states of stages 2 and 3 of a step).
// uni_mode: 0 the test streams the state and writes the RHS and a_max of the
// uniform subgrids; 1 (first stage of a step, whose combine takes those
// subgrids whole without reading their RHS) a_max only -- on a uniform level
// whose ghosts all have a source, from the interiors alone, since the state
// a step starts from has valid ghosts; 2 (stages 2 and 3 on a uniform
// level) the flags from the record of the combine before, nothing written
// for those subgrids.
static oct_status launch_rhs(oct_hydro *h, const double *U, double *dUdt, cudaStream_t st, int uni_slot = 0,
                             int uni_mode = 0)
{
    RhsArgs A;
    A.U = U;
    A.dUdt = dUdt;
    A.amax_tile = h->d_amax_tile;
    A.edge = h->d_edge;
    A.off = h->d_off;
    A.doff = h->d_doff;
    A.dx = h->d_dx;
    A.items = h->d_items;
    A.n_items = (int)h->items.size();
    A.nf = h->nf;
    A.gamma = h->gamma;
    A.eps1 = h->eps1;
    A.inv_gm1 = 1.0 / (h->gamma - 1.0);
    A.flags = h->d_flags;
    if (h->recon == OCT_RECON_PRIMITIVE) {
        if (!h->d_Wprim)
            return fail(OCT_E_STATE, "no buffer for the primitive variables");
        prim_cells_kernel<<<h->n_sub, 256, 0, st>>>(U, h->d_Wprim, h->d_edge, h->d_off, h->nf, h->gamma, h->eps1,
                                                    h->d_flags);
        CUDA_TRY(cudaGetLastError());
        A.U = h->d_Wprim;
    }
    const bool reflux = h->bc == OCT_BC_AMR && h->n_corr_cells > 0;
    A.faces = reflux ? h->d_faces : nullptr;
    A.face_slot = reflux ? h->d_face_slot : nullptr;
    A.order = h->d_order;
    A.ticket = h->d_ticket;
    A.sub_uniform = nullptr;
    A.field_uni = nullptr;
    const int form = form_of(h), mode = h->tile_mode;
    if (h->items_mode != mode || h->items_grid != grid_ctas(h))
        return fail(OCT_E_STATE, "work items were cut for another launch shape");
    h->uni_test = h->recon != OCT_RECON_PRIMITIVE && !reflux;
    if (h->uni_test) {
        // subgrids whose ghosted block is one value per field: skipped by the
        // RHS kernel
        int *flags = h->d_sub_uniform + (size_t)uni_slot * h->n_sub;
        // and, in FP64, the fields of each subgrid left that hold one value
        // (the RHS kernel reconstructs only the others)
        if (h->precision == 0)
            A.field_uni = h->d_field_uni;
        if (uni_mode == 2 && record_test_ok(h)) {
            // "yes" from the record; the other subgrids streamed
            CUDA_TRY(record_test_launch(h->precision, h->n_sub, st, A, h->d_nbr, h->d_out_uni, h->d_out_val, flags,
                                        nullptr));
            CUDA_TRY(uniform_launch(h->precision, h->n_sub, st, A, h->d_item_begin, flags, false, true));
        } else if (uni_mode == 1 && record_test_ok(h)) {
            CUDA_TRY(interior_record_launch(h->n_sub, st, A, h->d_u_uni, h->d_u_val));
            CUDA_TRY(record_test_launch(h->precision, h->n_sub, st, A, h->d_nbr, h->d_u_uni, h->d_u_val, flags,
                                        h->d_item_begin));
            CUDA_TRY(uniform_launch(h->precision, h->n_sub, st, A, h->d_item_begin, flags, false, true));
        } else {
            CUDA_TRY(uniform_launch(h->precision, h->n_sub, st, A, h->d_item_begin, flags, uni_mode == 0));
        }
        A.sub_uniform = flags;
    }
    A.live_items = nullptr;
    A.live_slot = nullptr;
    A.n_live = nullptr;
    int grid = std::min<int>(A.n_items, grid_ctas(h));
    if (h->uni_test && live_ok(h)) {
        // the items of the subgrids left, the last round cut in half when at
        // most half full
        CUDA_TRY(live_items_launch(h->n_sub, st, A.sub_uniform, h->d_item_begin, h->d_items, grid, h->items_live_split,
                                   h->d_live_items, h->d_live_slot, h->d_n_live, h->d_amax_tile));
        A.live_items = h->d_live_items;
        A.live_slot = h->d_live_slot;
        A.n_live = h->d_n_live;
    }
    CUDA_TRY(rhs_launch(form, mode, grid, st, A));
    CUDA_TRY(cudaGetLastError());
    if (reflux) {
        reflux_kernel<<<(h->n_corr_cells + 127) / 128, 128, 0, st>>>(dUdt, h->d_faces, h->d_corr, h->d_corr_first,
                                                                     h->n_corr_cells, h->nf, h->edge[0], h->d_dx);
        CUDA_TRY(cudaGetLastError());
    }
    return OCT_OK;
}

static oct_status ensure_scratch(oct_hydro *h)
{
    if (!h->d_L)
        CUDA_TRY(cudaMalloc(&h->d_L, sizeof(double) * std::max<long long>(1, h->rhs_len)));
    if (!h->d_W)
        CUDA_TRY(cudaMalloc(&h->d_W, sizeof(double) * std::max<long long>(1, h->state_len)));
    return OCT_OK;
}

extern "C" oct_status oct_hydro_rhs(oct_hydro_t h, const double *U, double *dUdt, double *amax, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_rhs");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U, "U")) != OCT_OK || (st = check_ptr(dUdt, "dUdt")) != OCT_OK)
        return st;
    const char *u0 = (const char *)U, *u1 = u0 + h->state_len * 8;
    const char *d0 = (const char *)dUdt, *d1 = d0 + h->rhs_len * 8;
    if (u0 < d1 && d0 < u1)
        return fail(OCT_E_ARG, "U and dUdt overlap");
    if ((st = sync_items(h)) != OCT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if ((st = launch_rhs(h, U, dUdt, s)) != OCT_OK)
        return st;
    if (amax) {
        amax_subgrid_kernel<<<(h->n_sub + 255) / 256, 256, 0, s>>>(h->n_sub, h->d_item_begin, h->d_amax_tile, amax);
        CUDA_TRY(cudaGetLastError());
    }
    return OCT_OK;
}

static oct_status launch_dt(oct_hydro *h, cudaStream_t s, bool capped = true)
{
    const int n = (int)h->items.size();
    const int grid = std::max(1, std::min(DT_MAX_BLOCKS, (n + DT_THREADS - 1) / DT_THREADS));
    dt_blocks_kernel<<<grid, DT_THREADS, 0, s>>>(n, h->d_items, h->d_dx, h->d_amax_tile, h->cfl,
                                                 capped ? h->d_dtcap : nullptr, h->d_dt_part, h->d_dt_count, h->d_dt);
    CUDA_TRY(cudaGetLastError());
    return OCT_OK;
}

extern "C" oct_status oct_hydro_max_dt(oct_hydro_t h, const double *U, double *dt_host_out, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_max_dt");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U, "U")) != OCT_OK)
        return st;
    if (!dt_host_out)
        return fail(OCT_E_ARG, "dt_host_out is NULL");
    if ((st = ensure_scratch(h)) != OCT_OK)
        return st;
    if ((st = sync_items(h)) != OCT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if ((st = launch_rhs(h, U, h->d_L, s)) != OCT_OK)
        return st;
    st = launch_dt(h, s, false);
    if (st != OCT_OK)
        return st;
    CUDA_TRY(cudaMemcpyAsync(dt_host_out, h->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return OCT_OK;
}

// changed: per-subgrid flags of the combine just before (null: fill all).
static oct_status launch_ghosts(oct_hydro *h, double *U, cudaStream_t s, const int *changed = nullptr)
{
    if (h->bc == OCT_BC_GIVEN)
        return OCT_OK;
    if (h->bc == OCT_BC_AMR) {
        amr_ghost_kernel<<<h->n_sub, 256, 0, s>>>(U, h->edge[0], h->d_off, h->nf, h->d_amr_plan, 0);
        CUDA_TRY(cudaGetLastError());
        if (h->has_prolong) {  // prolongations read the coarse blocks' ghosts of the first pass
            amr_ghost_kernel<<<h->n_sub, 256, 0, s>>>(U, h->edge[0], h->d_off, h->nf, h->d_amr_plan, 1);
            CUDA_TRY(cudaGetLastError());
        }
        return OCT_OK;
    }
    ghost_fill_kernel<<<h->n_sub, 256, 0, s>>>(U, h->edge[0], h->d_off, h->nf, h->d_nbr, h->d_flags, changed);
    CUDA_TRY(cudaGetLastError());
    return OCT_OK;
}

extern "C" oct_status oct_hydro_fill_ghosts(oct_hydro_t h, double *U, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_fill_ghosts");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U, "U")) != OCT_OK)
        return st;
    return launch_ghosts(h, U, (cudaStream_t)cuda_stream);
}

static oct_status launch_combine(oct_hydro *h, int stage, const double *U0, const double *X, double *out,
                                 cudaStream_t s)
{
    CombineArgs A;
    A.stage = stage;
    A.U0 = U0;
    A.X = X;
    A.out = out;
    A.L = h->d_L;
    A.dt = h->d_dt;
    A.edge = h->d_edge;
    A.off = h->d_off;
    A.doff = h->d_doff;
    A.nf = h->nf;
    A.gamma = h->gamma;
    A.rho_floor = h->rho_floor;
    A.eps2 = h->eps2;
    A.flags = h->d_flags;
    // the uniform flags of this stage's RHS inputs (stage 1: U; stages 2 and
    // 3: the stage state, and U as of stage 1), when the RHS ran that test
    A.uni_u0 = h->uni_test ? h->d_sub_uniform : nullptr;
    A.uni_x = h->uni_test ? h->d_sub_uniform + (stage == 1 ? 0 : h->n_sub) : nullptr;
    A.out_is_x = out == X;
    A.out_is_u0 = out == U0;
    // stages 1 and 2 record W for the next stage's uniform test; stage 1
    // also compares with the record of W that the last step left
    const bool rec = stage <= 2 && w_record_ok(h);
    A.out_uni = rec ? h->d_out_uni : nullptr;
    A.out_val = rec ? h->d_out_val : nullptr;
    A.changed = stage == 1 && !rec ? nullptr : h->d_changed;
    // persistent grid over whole subgrids (two cells a thread for edge 8)
    const int n_items = h->n_sub;
    const int grid = std::min(n_items, h->n_sm * h->combine_ctas[stage == 1 ? 1 : 0]);
    if (stage == 1)
        combine_kernel<true><<<(unsigned)grid, COMBINE_THREADS, 0, s>>>(A, n_items);
    else
        combine_kernel<false><<<(unsigned)grid, COMBINE_THREADS, 0, s>>>(A, n_items);
    CUDA_TRY(cudaGetLastError());
    return OCT_OK;
}

// The launches of one SSP-RK3 step on U (W: stage state, L: RHS register).
static oct_status enqueue_step(oct_hydro *h, double *U, cudaStream_t s)
{
    oct_status st;
    double *W = h->d_W;
    if (h->bc == OCT_BC_GIVEN)
        CUDA_TRY(cudaMemcpyAsync(W, U, sizeof(double) * h->state_len, cudaMemcpyDeviceToDevice, s));
    if ((st = launch_rhs(h, U, h->d_L, s, 0, 1)) != OCT_OK) return st;
    if ((st = launch_dt(h, s)) != OCT_OK) return st;
    // the ghost fills leave alone the subgrids whose neighbourhood the
    // combine before did not change: W's ghosts are valid after the last
    // step's stage 2 (and after stage 1's fill), U's on entry
    if (!w_record_ok(h))
        CUDA_TRY(cudaMemsetAsync(h->d_out_uni, 0, sizeof(int) * std::max(1, h->n_sub), s));
    if ((st = launch_combine(h, 1, U, U, W, s)) != OCT_OK) return st;
    if ((st = launch_ghosts(h, W, s, w_record_ok(h) ? h->d_changed : nullptr)) != OCT_OK) return st;
    if ((st = launch_rhs(h, W, h->d_L, s, 1, 2)) != OCT_OK) return st;
    if ((st = launch_combine(h, 2, U, W, W, s)) != OCT_OK) return st;
    if ((st = launch_ghosts(h, W, s, h->d_changed)) != OCT_OK) return st;
    if ((st = launch_rhs(h, W, h->d_L, s, 1, 2)) != OCT_OK) return st;
    if ((st = launch_combine(h, 3, U, W, U, s)) != OCT_OK) return st;
    if ((st = launch_ghosts(h, U, s, h->d_changed)) != OCT_OK) return st;
    return OCT_OK;
}

// Ghost-fill launches per stage.
static int per_fill_of(const oct_hydro *h)
{
    if (h->bc == OCT_BC_AMR)
        return h->has_prolong ? 2 : 1;
    return h->bc != OCT_BC_GIVEN ? 1 : 0;
}

extern "C" int oct_hydro_step_launches(oct_hydro_t h)
{
    if (!h || !h->layout_ok)
        return -1;
    const bool reflux = h->bc == OCT_BC_AMR && h->n_corr_cells > 0;
    // per stage the RHS kernel, with the primitive pass before it (primitive
    // reconstruction) or else the whole-subgrid uniform test and the work
    // list after it, and the flux correction after it across levels; the
    // uniform test is one streaming kernel, or on a uniform level whose
    // ghosts all have a source three (first stage: the interiors' record, the
    // test from it, the stream over the rest) and two (later stages: the test
    // from the combine's record, the stream over the rest)
    const bool uni = h->recon != OCT_RECON_PRIMITIVE && !reflux;
    const bool rec = uni && (h->bc == OCT_BC_PERIODIC || h->bc == OCT_BC_OUTFLOW) && h->ghosts_sourced;
    const int tests = uni ? (rec ? 3 + 2 + 2 : 3) : 0;
    const int extra = h->recon == OCT_RECON_PRIMITIVE ? 3 : (reflux ? 3 : 0);
    return 3 + tests + extra + (uni && live_ok(h) ? 3 : 0) + 1 + 3 + 3 * per_fill_of(h);
}

extern "C" oct_status oct_hydro_rk_step(oct_hydro_t h, double *U, double *dt_used_host_out, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_rk_step");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U, "U")) != OCT_OK)
        return st;
    if ((st = ensure_scratch(h)) != OCT_OK)
        return st;
    if ((st = sync_items(h)) != OCT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (h->graphs.size() >= 16 && !h->graphs.count(U))
        drop_graphs(h);  // bound the per-state-pointer graph cache
    GraphEntry &ge = h->graphs[U];
    if (!ge.exec && s != 0) {
        cudaGraph_t graph;
        CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = enqueue_step(h, U, s);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st != OCT_OK)
            return st;
        if (e != cudaSuccess)
            return fail(OCT_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ge.exec = nullptr;
            return fail(OCT_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        }
    }
    if (ge.exec) {
        CUDA_TRY(cudaGraphLaunch(ge.exec, s));
    } else if ((st = enqueue_step(h, U, s)) != OCT_OK) {
        return st;
    }
    if (dt_used_host_out) {
        CUDA_TRY(cudaMemcpyAsync(dt_used_host_out, h->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return OCT_OK;
}

// Whether the host-buffer step may copy in only the interior z-planes of each
// field block and refill the ghosts on the device: a uniform level (the
// ghosts are copies of interior cells, which the step requires of its input
// anyway) in the default contiguous layout (subgrid s at s nf B^3, so that
// the runs to copy are evenly spaced and one 2D copy takes them all).
static bool interior_copy_ok(const oct_hydro *h)
{
    if (!(h->bc == OCT_BC_PERIODIC || h->bc == OCT_BC_OUTFLOW) || !h->ghosts_sourced || h->edge.empty())
        return false;
    const long long B = h->edge[0] + 2 * NG, block = (long long)h->nf * B * B * B;
    for (int s = 0; s < h->n_sub; s++)
        if (h->edge[s] != h->edge[0] || h->off[s] != s * block)
            return false;
    return true;
}

extern "C" oct_status oct_hydro_host_copy_bytes(oct_hydro_t h, int64_t *h2d_bytes, int64_t *d2h_bytes)
{
    if (!h || !h->layout_ok)
        return fail(OCT_E_ARG, "handle is NULL or has no layout");
    const long long full = (long long)sizeof(double) * h->state_len;
    long long in = full;
    if (interior_copy_ok(h)) {
        const long long E = h->edge[0], B = E + 2 * NG;
        in = (long long)sizeof(double) * h->n_sub * h->nf * E * B * B;
    }
    if (h2d_bytes)
        *h2d_bytes = in;
    if (d2h_bytes)
        *d2h_bytes = full;
    return OCT_OK;
}

extern "C" oct_status oct_hydro_rk_steps_host(oct_hydro_t h, double *U_host, int n_steps, double *dt_last_out,
                                              void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_rk_steps_host");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if (!U_host)
        return fail(OCT_E_ARG, "U_host is NULL");
    if (n_steps < 0)
        return fail(OCT_E_ARG, "n_steps must be >= 0");
    if (!h->d_Uhost)
        CUDA_TRY(cudaMalloc(&h->d_Uhost, sizeof(double) * h->state_len));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    size_t bytes = sizeof(double) * h->state_len;
    if (interior_copy_ok(h)) {
        // the interior z-planes of every field block (one evenly spaced run
        // each), then the ghosts from the interiors on the device
        const size_t E = h->edge[0], B = E + 2 * NG, B2 = B * B;
        const size_t pitch = sizeof(double) * B2 * B;
        CUDA_TRY(cudaMemcpy2DAsync(h->d_Uhost + NG * B2, pitch, U_host + NG * B2, pitch, sizeof(double) * E * B2,
                                   (size_t)h->n_sub * h->nf, cudaMemcpyHostToDevice, s));
        if ((st = launch_ghosts(h, h->d_Uhost, s)) != OCT_OK)
            return st;
    } else {
        CUDA_TRY(cudaMemcpyAsync(h->d_Uhost, U_host, bytes, cudaMemcpyHostToDevice, s));
    }
    for (int i = 0; i < n_steps; i++)
        if ((st = oct_hydro_rk_step(h, h->d_Uhost, nullptr, cuda_stream)) != OCT_OK)
            return st;
    CUDA_TRY(cudaMemcpyAsync(U_host, h->d_Uhost, bytes, cudaMemcpyDeviceToHost, s));
    if (dt_last_out)
        CUDA_TRY(cudaMemcpyAsync(dt_last_out, h->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return OCT_OK;
}

extern "C" oct_status oct_hydro_rhs_host(oct_hydro_t h, const double *U_host, double *dUdt_host, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_rhs_host");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if (!U_host || !dUdt_host)
        return fail(OCT_E_ARG, "host buffer is NULL");
    if (!h->d_Uhost)
        CUDA_TRY(cudaMalloc(&h->d_Uhost, sizeof(double) * h->state_len));
    if (!h->d_Lhost)
        CUDA_TRY(cudaMalloc(&h->d_Lhost, sizeof(double) * std::max<long long>(1, h->rhs_len)));
    if ((st = sync_items(h)) != OCT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CUDA_TRY(cudaMemcpyAsync(h->d_Uhost, U_host, sizeof(double) * h->state_len, cudaMemcpyHostToDevice, s));
    if ((st = launch_rhs(h, h->d_Uhost, h->d_Lhost, s)) != OCT_OK)
        return st;
    CUDA_TRY(cudaMemcpyAsync(dUdt_host, h->d_Lhost, sizeof(double) * h->rhs_len, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return OCT_OK;
}

// Autotuner cache (optional): when the environment variable
// OCT_HYDRO_TUNE_CACHE names a file, a tuning result is looked up there
// before any trial launch and appended after one.  One line per result:
// "<key> <tile mode> <CTAs per SM>", the key made of the GPU name, its SM
// count, the form (precision, reconstruction), the field count and the
// batch's edge counts, e.g. "NVIDIA_GB300|152|f0|nf11|e8x512 1 2".
static std::mutex g_tune_mutex;

static std::string tune_key(const oct_hydro *h)
{
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, h->device) == cudaSuccess ? prop.name : "gpu";
    for (char &c : name)
        if (c == ' ' || c == '|')
            c = '_';
    int n8 = 0, n12 = 0, n16 = 0;
    for (int E : h->edge)
        (E == 8 ? n8 : (E == 12 ? n12 : n16))++;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|f%d|nf%d|e8x%d,e12x%d,e16x%d", name.c_str(), h->n_sm, h->precision + 2 * h->recon,
             h->nf, n8, n12, n16);
    return buf;
}

static bool tune_lookup(const std::string &key, int *mode, int *use)
{
    const char *path = getenv("OCT_HYDRO_TUNE_CACHE");
    if (!path || !*path)
        return false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE *f = fopen(path, "r");
    if (!f)
        return false;
    char k[256];
    int m, u;
    bool found = false;
    while (fscanf(f, "%255s %d %d", k, &m, &u) == 3)
        if (key == k && m >= 0 && m < RHS_MODES && u >= 1) {
            *mode = m, *use = u, found = true;  // the last entry for a key wins
        }
    fclose(f);
    return found;
}

static void tune_store(const std::string &key, int mode, int use)
{
    const char *path = getenv("OCT_HYDRO_TUNE_CACHE");
    if (!path || !*path)
        return;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE *f = fopen(path, "a");
    if (!f)
        return;  // a cache that cannot be written is not an error
    fprintf(f, "%s %d %d\n", key.c_str(), mode, use);
    fclose(f);
}

extern "C" oct_status oct_hydro_autotune(oct_hydro_t h, const double *U_sample, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_autotune");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U_sample, "U_sample")) != OCT_OK)
        return st;
    if ((st = ensure_scratch(h)) != OCT_OK)
        return st;
    const std::string key = tune_key(h);
    {
        int mode, use;
        if (tune_lookup(key, &mode, &use) && mode < RHS_MODES && use <= h->ctas_per_sm[form_of(h)][mode]) {
            h->tile_mode = mode;
            h->cta_use[form_of(h)][mode] = use;
            return sync_items(h);
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // candidates: tile shape (threads per subgrid) x resident CTAs per SM of
    // the persistent grid; each timed on 2 launches after one untimed
    float best = 1e30f;
    const int prec = form_of(h);
    int best_mode = h->tile_mode, best_use = h->cta_use[prec][h->tile_mode];
    for (int mode = 0; mode < RHS_MODES; mode++) {
        if (h->ctas_per_sm[prec][mode] < 1)
            continue;  // this launch shape does not fit with this field count
        h->tile_mode = mode;
        for (int use = 1; use <= h->ctas_per_sm[prec][mode]; use++) {
            h->cta_use[prec][mode] = use;
            // the items are cut for this grid
            if ((st = sync_items(h)) != OCT_OK)
                return st;
            float tot = 0.0f;
            for (int rep = 0; rep < 3; rep++) {
                CUDA_TRY(cudaEventRecord(e0, s));
                if ((st = launch_rhs(h, U_sample, h->d_L, s)) != OCT_OK)
                    return st;
                CUDA_TRY(cudaEventRecord(e1, s));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0)
                    tot += ms;
            }
            if (tot < best) {
                best = tot;
                best_mode = mode;
                best_use = use;
            }
        }
        h->cta_use[prec][mode] = 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tile_mode = best_mode;
    h->cta_use[prec][best_mode] = best_use;
    tune_store(key, best_mode, best_use);
    return sync_items(h);
}

extern "C" oct_status oct_hydro_launch_info(oct_hydro_t h, int *tile_mode, int *ctas_per_sm, int *n_items)
{
    DeviceGuard device_guard(h);
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if (tile_mode)
        *tile_mode = h->tile_mode;
    if (ctas_per_sm) {
        const int use = h->cta_use[form_of(h)][h->tile_mode];
        *ctas_per_sm = use > 0 ? use : h->ctas_per_sm[form_of(h)][h->tile_mode];
    }
    if (n_items)
        *n_items = (int)h->items.size();
    return OCT_OK;
}

extern "C" oct_status oct_hydro_get_error_flags(oct_hydro_t h, uint32_t *flags)
{
    DeviceGuard device_guard(h);
    if (!h || !flags)
        return fail(OCT_E_ARG, "handle or flags is NULL");
    unsigned v = 0;
    CUDA_TRY(cudaMemcpy(&v, h->d_flags, sizeof v, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(h->d_flags, 0, sizeof v));
    *flags = v;
    return OCT_OK;
}

extern "C" const char *oct_hydro_last_error(void)
{
    return g_last_error.c_str();
}

extern "C" void oct_hydro_destroy(oct_hydro_t h)
{
    DeviceGuard device_guard(h);
    if (!h)
        return;
    free_layout(h);
    dfree(h->d_flags);
    dfree(h->d_dt);
    dfree(h->d_dtcap);
    dfree(h->d_dt_part);
    dfree(h->d_dt_count);
    dfree(h->d_ticket);
    dfree(h->d_gst_off);
    dfree(h->d_gst_k);
    delete h;
}

// Raises the monopole kernel's dynamic shared-memory limit on the current
// device to at least bytes (never lowers it: other handles may need more).
static cudaError_t monopole_smem_limit(size_t bytes)
{
    static std::mutex mu;
    static size_t set_to[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64)
        return e != cudaSuccess ? e : cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (bytes <= set_to[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(monopole_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        set_to[dev] = bytes;
    return e;
}

extern "C" oct_status oct_hydro_gravity_monopole(oct_hydro_t h, const double *U, double G, double r_s, double *phi,
                                                 double *g, void *cuda_stream)
{
    DeviceGuard device_guard(h);
    NvtxRange nvtx_range("oct_hydro_gravity_monopole");
    oct_status st = check_ready(h);
    if (st != OCT_OK)
        return st;
    if ((st = check_ptr(U, "U")) != OCT_OK || (st = check_ptr(phi, "phi")) != OCT_OK ||
        (st = check_ptr(g, "g")) != OCT_OK)
        return st;
    if (h->bc != OCT_BC_PERIODIC && h->bc != OCT_BC_OUTFLOW)
        return fail(OCT_E_STATE, "gravity needs one level with a neighbour table (periodic or outflow layout)");
    const int E = h->edge[0];
    for (int s = 1; s < h->n_sub; s++)
        if (h->dx[s] != h->dx[0])
            return fail(OCT_E_ARG, "gravity needs one cell width for every subgrid (subgrid %d differs)", s);
    if (!(G > 0.0) || !std::isfinite(G))
        return fail(OCT_E_ARG, "G must be positive and finite (got %g)", G);
    if (!(r_s >= 1.0) || !std::isfinite(r_s) || (int)std::floor(r_s) > E)
        return fail(OCT_E_ARG, "r_s must be in [1, edge] cell widths (got %g)", r_s);
    const int R = (int)std::floor(r_s);
    const int S = E + 2 * R;
    if (r_s != h->gst_rs || S != h->gst_S) {
        // the stencil: offsets with 0 < |d|^2 <= r_s^2, z outermost, then y, then x
        std::vector<int> off;
        std::vector<GravEntry> k;
        const double r2max = r_s * r_s;
        for (int dz = -R; dz <= R; dz++)
            for (int dy = -R; dy <= R; dy++)
                for (int dxx = -R; dxx <= R; dxx++) {
                    const double d2 = (double)(dxx * dxx + dy * dy + dz * dz);
                    if (d2 == 0.0 || d2 > r2max)
                        continue;
                    const double r = std::sqrt(d2), r3 = d2 * r;
                    off.push_back((dz * S + dy) * S + dxx);
                    k.push_back(GravEntry{1.0 / r, dxx / r3, dy / r3, dz / r3});
                }
        dfree(h->d_gst_off);
        dfree(h->d_gst_k);
        h->gst_rs = 0.0;
        CUDA_TRY(cudaMalloc(&h->d_gst_off, sizeof(int) * off.size()));
        CUDA_TRY(cudaMalloc(&h->d_gst_k, sizeof(GravEntry) * k.size()));
        CUDA_TRY(cudaMemcpy(h->d_gst_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->d_gst_k, k.data(), sizeof(GravEntry) * k.size(), cudaMemcpyHostToDevice));
        h->gst_n = (int)off.size();
        h->gst_rs = r_s;
        h->gst_S = S;
    }
    const size_t smem = monopole_smem(S, h->gst_n);
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (smem > (size_t)optin)
        return fail(OCT_E_ARG, "r_s = %g needs %zu bytes of shared memory for edge %d (at most %d)", r_s, smem, E,
                    optin);
    CUDA_TRY(monopole_smem_limit(smem));
    const double dx = h->dx[0];
    monopole_kernel<<<h->n_sub, MONO_THREADS, smem, (cudaStream_t)cuda_stream>>>(
        U, h->d_off, E, h->d_nbr, R, h->gst_n, h->d_gst_off, h->d_gst_k, dx * dx * dx, -G / dx, G / (dx * dx), phi, g);
    CUDA_TRY(cudaGetLastError());
    return OCT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free RHS + dt entry point.
//
// For callers that cannot call cudaMalloc on their hot path: host programs
// whose device memory is all handed out by their own pool allocator (a
// cudaMalloc there fails or fragments the pool), and programs that must not
// take the implicit device-wide synchronisation that cudaMalloc/cudaFree can
// cause.  Everything the RHS and dt kernels need beyond the caller's inputs
// and outputs lives in one file-scope device array of fixed size, reserved
// when the library is loaded on a device and kept until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int NA_MAX_SUB = 4096;              // largest batch the static scratch holds
constexpr int NA_MAX_ITEMS = 4 * NA_MAX_SUB;  // at most 4 work items per subgrid (edge 12 or 16)
constexpr size_t NA_FLAGS = 0;
constexpr size_t NA_EDGE = 256;
constexpr size_t NA_OFF = NA_EDGE + sizeof(int) * NA_MAX_SUB;
constexpr size_t NA_DOFF = NA_OFF + sizeof(long long) * NA_MAX_SUB;
constexpr size_t NA_ITEMS = NA_DOFF + sizeof(long long) * NA_MAX_SUB;
constexpr size_t NA_AMAX = NA_ITEMS + sizeof(WorkItem) * NA_MAX_ITEMS;
constexpr size_t NA_BYTES = NA_AMAX + sizeof(double) * NA_MAX_ITEMS;  // 475,392 bytes
static_assert(NA_ITEMS % 16 == 0 && NA_OFF % 8 == 0 && NA_AMAX % 8 == 0, "scratch sub-array alignment");
}  // namespace

// The static scratch: flag word, per-subgrid edge / state offset / RHS
// offset, the work list and the per-item signal speeds.  In host code this
// name is only a stand-in for the device array; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch
    int n_sm = 0;
    int ctas[2] = {0, 0};
};
static NoallocDevice g_noalloc[64];
static std::mutex g_noalloc_mutex;

// Packed uniform layout and work list of a batch, written into the static
// scratch: block s at s * round4(nf * (E+6)^3), RHS at s * nf * E^3, tiles as
// in the handle's default work list.
__global__ void noalloc_layout_kernel(int n_sub, int E, int nf, int *edge, long long *off, long long *doff,
                                      WorkItem *items)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub)
        return;
    long long B = E + 2 * NG;
    long long len = (nf * B * B * B + 3) / 4 * 4;
    edge[s] = E;
    off[s] = s * len;
    doff[s] = (long long)s * nf * E * E * E;
    int t = (E == 12) ? 6 : 8;
    int per_row = E / t;
    for (int k = 0; k < per_row * per_row; k++) {
        WorkItem w;
        w.s = s;
        w.x0 = (k % per_row) * t;
        w.y0 = (k / per_row) * t;
        w.txty = t | (t << 8);
        items[s * per_row * per_row + k] = w;
    }
}

// Once per device, with that device current: the scratch address, the line
// tables and the RHS kernels' launch attributes.
static oct_status noalloc_setup(int dev, NoallocDevice **out)
{
    if (dev < 0 || dev >= 64)
        return fail(OCT_E_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice &d = g_noalloc[dev];
    if (!d.ready) {
        void *p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        CUDA_TRY(cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev));
        for (int prec = 0; prec < 2; prec++) {
            int nb = 0;
            CUDA_TRY(rhs_prepare(prec, 0, MAXNF, &nb));
            if (nb < 1)
                return fail(OCT_E_CUDA, "RHS kernel does not fit on an SM");
            d.ctas[prec] = nb;
        }
        d.base = (unsigned char *)p;
        d.ready = true;
    }
    *out = &d;
    return OCT_OK;
}

extern "C" oct_status oct_hydro_rhs_dt_noalloc(int n_subgrids, int edge, int n_species, double gamma, int precision,
                                               double cfl, double de_switch1, const double *U, const double *dx,
                                               double *dUdt, double *dt, void *cuda_stream)
{
    NvtxRange nvtx_range("oct_hydro_rhs_dt_noalloc");
    if (n_subgrids <= 0 || n_subgrids > NA_MAX_SUB)
        return fail(OCT_E_ARG,
                    "n_subgrids must be in 1..%d, the size of the static scratch of the allocation-free call "
                    "(got %d)",
                    NA_MAX_SUB, n_subgrids);
    if (!valid_edge(edge))
        return fail(OCT_E_ARG, "edge must be 8, 12 or 16 (got %d)", edge);
    if (n_species < 0 || n_species > MAXNF - 6)
        return fail(OCT_E_ARG, "n_species must be in 0..%d (got %d)", MAXNF - 6, n_species);
    if (!(gamma > 1.0) || !std::isfinite(gamma))
        return fail(OCT_E_ARG, "gamma must be > 1 (got %g)", gamma);
    if (precision != OCT_FP64 && precision != OCT_MIXED)
        return fail(OCT_E_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (!(cfl > 0.0 && cfl <= 1.0))
        return fail(OCT_E_ARG, "cfl must be in (0, 1] (got %g)", cfl);
    if (!(de_switch1 >= 0.0 && de_switch1 < 1.0))
        return fail(OCT_E_ARG, "de_switch1 must be in [0, 1)");
    oct_status st;
    if ((st = check_ptr(U, "U")) != OCT_OK || (st = check_ptr(dUdt, "dUdt")) != OCT_OK)
        return st;
    if (!dx || !dt)
        return fail(OCT_E_ARG, "dx and dt must not be NULL");
    const int nf = 6 + n_species;
    const long long B = edge + 2 * NG;
    const long long state_len = (long long)n_subgrids * ((nf * B * B * B + 3) / 4 * 4);
    const long long rhs_len = (long long)n_subgrids * nf * edge * edge * edge;
    const char *u0 = (const char *)U, *u1 = u0 + state_len * 8;
    const char *d0 = (const char *)dUdt, *d1 = d0 + rhs_len * 8;
    if (u0 < d1 && d0 < u1)
        return fail(OCT_E_ARG, "U and dUdt overlap");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    NoallocDevice *D = nullptr;
    if ((st = noalloc_setup(dev, &D)) != OCT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char *base = D->base;
    const int per = (edge == 8) ? 1 : 4;
    const int n_items = n_subgrids * per;
    unsigned *flags = (unsigned *)(base + NA_FLAGS);
    int *d_edge = (int *)(base + NA_EDGE);
    long long *d_off = (long long *)(base + NA_OFF);
    long long *d_doff = (long long *)(base + NA_DOFF);
    WorkItem *d_items = (WorkItem *)(base + NA_ITEMS);
    double *d_amax = (double *)(base + NA_AMAX);
    // the flag word is the only part that has to start at zero; every other
    // entry is rewritten below before it is read
    CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
    noalloc_layout_kernel<<<(n_subgrids + 127) / 128, 128, 0, s>>>(n_subgrids, edge, nf, d_edge, d_off, d_doff,
                                                                     d_items);
    CUDA_TRY(cudaGetLastError());
    RhsArgs A;
    A.U = U;
    A.dUdt = dUdt;
    A.amax_tile = d_amax;
    A.edge = d_edge;
    A.off = d_off;
    A.doff = d_doff;
    A.dx = dx;
    A.items = d_items;
    A.n_items = n_items;
    A.nf = nf;
    A.gamma = gamma;
    A.eps1 = de_switch1;
    A.flags = flags;
    A.inv_gm1 = 1.0 / (gamma - 1.0);
    A.faces = nullptr;
    A.face_slot = nullptr;
    A.order = nullptr;
    A.ticket = nullptr;
    A.sub_uniform = nullptr;  // the kernel's own per-item uniform test
    A.field_uni = nullptr;
    A.live_items = nullptr;
    A.live_slot = nullptr;
    A.n_live = nullptr;
    int grid = std::min(n_items, D->n_sm * D->ctas[precision]);
    CUDA_TRY(rhs_launch(precision, 0, grid, s, A));
    dt_kernel<<<1, 1024, 0, s>>>(n_items, d_items, dx, d_amax, cfl, nullptr, dt);
    CUDA_TRY(cudaGetLastError());
    return OCT_OK;
}
