// C ABI of the batched runner (declared in include/lbm.h): many independent
// FP32 lattices, each an lbm_handle of its own, advanced together by the
// persistent batched kernel (lbm_batch_kernels.cuh) in one cooperative launch
// per call -- or per 32 steps, replayed from a captured CUDA graph -- with the
// tile shape chosen by timing candidates (lbm_batch_autotune).
#include "lbm.h"
#include "lbm_handle.h"
#include "lbm_internal.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr size_t BALIGN = 256;
constexpr int MIN_TILE_H = 4;
constexpr long long DEFAULT_SPIN_LIMIT = 1LL << 21;  // ~1 s of polling per wait
thread_local char g_batch_error[512] = "";

size_t balign_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Tiles of the finest tiling any call may choose (32 x MIN_TILE_H): the tables
// of the workspace are sized for it.
long long max_tiles(lbm_handle* const* cases, int n) {
    long long t = 0;
    for (int i = 0; i < n; ++i)
        t += (long long)((cases[i]->p.nx + 31) / 32) * ((cases[i]->p.ny + MIN_TILE_H - 1) / MIN_TILE_H);
    return t;
}

struct BatchLayout {
    size_t off_cases, off_tiles, off_nbr, off_done, off_status, total;
};

BatchLayout batch_layout(int ncases, long long tiles) {
    BatchLayout L;
    L.off_cases = 0;
    L.off_tiles = balign_up(L.off_cases + (size_t)ncases * sizeof(lbm::BatchCase), BALIGN);
    L.off_nbr = balign_up(L.off_tiles + (size_t)tiles * sizeof(lbm::BatchTile), BALIGN);
    L.off_done = balign_up(L.off_nbr + (size_t)tiles * lbm::BATCH_NEIGHBOURS * sizeof(int), BALIGN);
    L.off_status = balign_up(L.off_done + (size_t)tiles * sizeof(unsigned), BALIGN);
    L.total = L.off_status + BALIGN;
    return L;
}

// Checks shared by workspace sizing and creation.
int check_cases(lbm_handle* const* cases, int n, char* err, size_t len) {
    if (!cases || n < 1) { snprintf(err, len, "need at least one case"); return LBM_ERR_ARG; }
    for (int i = 0; i < n; ++i) {
        const lbm_handle* h = cases[i];
        if (!h) { snprintf(err, len, "case %d is NULL", i); return LBM_ERR_ARG; }
        if (h->p.precision != LBM_FP32) { snprintf(err, len, "case %d: the batched runner takes LBM_FP32 lattices", i); return LBM_ERR_ARG; }
        if (h->p.scalar_model != LBM_SCALAR_TWO || h->p.grad_scheme != LBM_GRAD_STENCIL) {
            snprintf(err, len, "case %d: the batched runner takes the two-scalar model with stencil gradients", i);
            return LBM_ERR_ARG;
        }
        if (h->p.scalar_q != cases[0]->p.scalar_q) { snprintf(err, len, "case %d: all cases must share scalar_q", i); return LBM_ERR_ARG; }
        if (h->device != cases[0]->device) { snprintf(err, len, "case %d: all cases must be on one device", i); return LBM_ERR_ARG; }
        if (h->stream != cases[0]->stream) { snprintf(err, len, "case %d: all cases must share one stream", i); return LBM_ERR_ARG; }
        for (int j = 0; j < i; ++j)
            if (cases[j] == h) { snprintf(err, len, "case %d repeats case %d", i, j); return LBM_ERR_ARG; }
    }
    return LBM_OK;
}

using Launch = cudaError_t (*)(const lbm::BatchArgs&, cudaStream_t);
using Occupancy = int (*)();

bool kernel_for(int q, int tile_w, Launch* launch, Occupancy* occ) {
#define LBM_PICK(Q, NW)                                 \
    if (q == Q && tile_w == 32 * NW) {                  \
        *launch = lbm::launch_batch<Q, NW>;             \
        *occ = lbm::batch_blocks_per_sm<Q, NW>;         \
        return true;                                    \
    }
    LBM_PICK(5, 1) LBM_PICK(5, 2) LBM_PICK(5, 4)
    LBM_PICK(9, 1) LBM_PICK(9, 2) LBM_PICK(9, 4)
#undef LBM_PICK
    return false;
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_handle*> cases;
    int device = 0;
    int q = 5;
    cudaStream_t stream = nullptr;
    uint8_t* ws = nullptr;
    BatchLayout L{};
    long long tiles_cap = 0;
    // current tiling
    int tile_w = 0, tile_h = 0, ntiles = 0, grid = 0;
    Launch launch = nullptr;
    int64_t steps = 0;          // steps since the counters were reset
    std::vector<int> cur0;      // buffer of each case at the reset
    long long spin_limit = DEFAULT_SPIN_LIMIT;
    int hold_tile = -1;
    bool failed = false;        // a wait gave up: the lattices are out of step
    cudaGraphExec_t graph = nullptr;
    bool graph_tried = false;
    // pinned staging of the case descriptors; the event marks the end of the
    // last copy out of it, so a reset rewrites it only once that copy is done
    lbm::BatchCase* h_cases = nullptr;
    cudaEvent_t cases_ev = nullptr;
    bool cases_ev_live = false;
    // side streams for the per-case work of the batch-level restart, field and
    // checkpoint calls: forked from and joined back into `stream` by events
    static constexpr int NSIDE = 8;
    cudaStream_t side[NSIDE] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[NSIDE] = {};
    int nside = 0;
    char err[512] = "";

    cudaError_t make_side_streams() {
        nside = (int)std::min<size_t>(NSIDE, cases.size());
        cudaError_t e = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
        for (int j = 0; j < nside && e == cudaSuccess; ++j) {
            e = cudaStreamCreateWithFlags(&side[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev[j], cudaEventDisableTiming);
        }
        return e;
    }

    void free_side_streams() {
        for (int j = 0; j < NSIDE; ++j) {
            if (side[j]) cudaStreamDestroy(side[j]);
            if (join_ev[j]) cudaEventDestroy(join_ev[j]);
            side[j] = nullptr;
            join_ev[j] = nullptr;
        }
        if (fork_ev) cudaEventDestroy(fork_ev);
        fork_ev = nullptr;
    }

    // op(i, s) issues case i's work on stream s; the cases are dealt round-robin
    // to the side streams, which start after everything queued on `stream` and
    // which `stream` waits for before anything issued after this call.
    template <typename Op>
    cudaError_t fan_out(Op&& op) {
        cudaError_t e = cudaEventRecord(fork_ev, stream);
        for (int j = 0; j < nside && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(side[j], fork_ev, 0);
        if (e != cudaSuccess) return e;
        for (size_t i = 0; i < cases.size() && e == cudaSuccess; ++i) e = op(i, side[i % nside]);
        for (int j = 0; j < nside; ++j) {
            cudaError_t r = cudaEventRecord(join_ev[j], side[j]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(stream, join_ev[j], 0);
            if (e == cudaSuccess) e = r;
        }
        return e;
    }

    lbm::BatchCase* d_cases() const { return reinterpret_cast<lbm::BatchCase*>(ws + L.off_cases); }
    lbm::BatchTile* d_tiles() const { return reinterpret_cast<lbm::BatchTile*>(ws + L.off_tiles); }
    int* d_nbr() const { return reinterpret_cast<int*>(ws + L.off_nbr); }
    unsigned* d_done() const { return reinterpret_cast<unsigned*>(ws + L.off_done); }
    unsigned* d_status() const { return reinterpret_cast<unsigned*>(ws + L.off_status); }

    int fail(int code, const char* what, cudaError_t e = cudaSuccess) {
        if (e != cudaSuccess) snprintf(err, sizeof(err), "%s: %s", what, cudaGetErrorString(e));
        else snprintf(err, sizeof(err), "%s", what);
        return code;
    }

    void drop_graph() {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        graph_tried = false;
    }

    lbm::BatchArgs args(int nsteps) const {
        lbm::BatchArgs a;
        a.cases = d_cases();
        a.tiles = d_tiles();
        a.nbr = d_nbr();
        a.done = d_done();
        a.status = d_status();
        a.ntiles = ntiles;
        a.nsteps = nsteps;
        a.spin_limit = spin_limit;
        a.hold_tile = hold_tile;
        a.grid = grid;
        return a;
    }

    // Case descriptors with each lattice's current buffer, step counters and
    // status word zeroed (stream-ordered after everything already queued; the
    // host does not wait for the stream).
    cudaError_t reset_counters() {
        if (cases_ev_live) {
            const cudaError_t w = cudaEventSynchronize(cases_ev);
            if (w != cudaSuccess) return w;
        }
        lbm::BatchCase* hc = h_cases;
        cur0.resize(cases.size());
        for (size_t i = 0; i < cases.size(); ++i) {
            lbm_handle* h = cases[i];
            lbm::BatchCase& c = hc[i];
            std::memset(&c, 0, sizeof(c));
            c.g = h->geo;
            c.C = h->cf;
            c.pop[0] = h->pop(0);
            c.pop[1] = h->pop(1);
            c.prev = h->prev();
            c.flag = h->flag();
            c.cur0 = h->cur;
            cur0[i] = h->cur;
        }
        cudaError_t e = cudaMemcpyAsync(d_cases(), hc, cases.size() * sizeof(lbm::BatchCase),
                                        cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaEventRecord(cases_ev, stream);
        cases_ev_live = e == cudaSuccess;
        if (e == cudaSuccess) e = cudaMemsetAsync(d_done(), 0, (size_t)tiles_cap * sizeof(unsigned), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_status(), 0, BALIGN, stream);
        steps = 0;
        failed = false;
        return e;
    }

    // A case stepped, re-initialised or restored on its own since the last reset
    // may hold its state in the other buffer: then the counters start over.
    cudaError_t resync_cases() {
        for (size_t i = 0; i < cases.size(); ++i)
            if (cases[i]->cur != ((cur0[i] + (int)(steps & 1)) & 1)) return reset_counters();
        return cudaSuccess;
    }

    cudaError_t launch_steps(int n) { return launch(args(n), stream); }

    // A graph of one GRAPH_STEPS-step launch; falls back to plain launches if the
    // cooperative launch cannot be captured.
    void try_graph() {
        graph_tried = true;
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return; }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = launch(args(lbm::detail::GRAPH_STEPS), cap);
            e = cudaStreamEndCapture(cap, &g);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess && g) e = cudaGraphInstantiate(&graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess && graph) {
            e = cudaGraphUpload(graph, stream);  // now, not at the first launch
            if (e != cudaSuccess) cudaGraphExecDestroy(graph);
        }
        if (e != cudaSuccess) { graph = nullptr; cudaGetLastError(); }
        cudaStreamDestroy(cap);
    }
};

namespace {

// Tiles of every case (row-major per case), their neighbour lists and the launch
// size for tile_w x tile_h.
int build_tiling(lbm_batch* b, int tile_w, int tile_h) {
    Launch launch;
    Occupancy occ;
    if (!kernel_for(b->q, tile_w, &launch, &occ)) return b->fail(LBM_ERR_ARG, "tile width must be 32, 64 or 128");
    if (tile_h < MIN_TILE_H) return b->fail(LBM_ERR_ARG, "tile height must be >= 4");
    std::vector<lbm::BatchTile> tiles;
    std::vector<int> nbr;
    // node coordinate a stencil or pull lands on: periodic wrap or wall clamp
    auto res = [](int v, int n, bool wall) {
        if (wall) return std::min(std::max(v, 0), n - 1);
        v %= n;
        return v < 0 ? v + n : v;
    };
    for (size_t c = 0; c < b->cases.size(); ++c) {
        const lbm_handle* h = b->cases[c];
        const int nx = h->p.nx, ny = h->p.ny;
        const int tx = (nx + tile_w - 1) / tile_w, ty = (ny + tile_h - 1) / tile_h;
        const int base = (int)tiles.size();
        const bool wx = h->p.bc_x == LBM_BC_WALL, wy = h->p.bc_y == LBM_BC_WALL;
        // A tile's step reads the populations of columns x0-2 .. x0+W+1 and rows
        // ya-2 .. yb+1 (its nodes, its halo ring and their upstream nodes), each
        // wrapped or clamped.  Tile columns / rows those reads fall in:
        std::vector<std::vector<int>> col_reach(tx), row_reach(ty);
        for (int i = 0; i < tx; ++i)
            for (int xx = i * tile_w - 2; xx <= i * tile_w + tile_w + 1; ++xx) {
                const int t = res(xx, nx, wx) / tile_w;
                if (std::find(col_reach[i].begin(), col_reach[i].end(), t) == col_reach[i].end())
                    col_reach[i].push_back(t);
            }
        for (int j = 0; j < ty; ++j)
            for (int yy = j * tile_h - 2; yy <= std::min(ny, (j + 1) * tile_h) + 1; ++yy) {
                const int t = res(yy, ny, wy) / tile_h;
                if (std::find(row_reach[j].begin(), row_reach[j].end(), t) == row_reach[j].end())
                    row_reach[j].push_back(t);
            }
        // A tile waits for every tile it reads (their previous step must be
        // complete) and for every tile that reads it (they must have finished
        // reading the buffer it is about to overwrite): the symmetric closure.
        std::vector<std::vector<int>> wait(tx * ty);
        for (int j = 0; j < ty; ++j)
            for (int i = 0; i < tx; ++i) {
                const int self = j * tx + i;
                for (int r : row_reach[j])
                    for (int q : col_reach[i]) {
                        const int o = r * tx + q;
                        if (o == self) continue;
                        wait[self].push_back(o);
                        wait[o].push_back(self);
                    }
            }
        for (int j = 0; j < ty; ++j)
            for (int i = 0; i < tx; ++i) {
                lbm::BatchTile t;
                t.c = (int)c;
                t.x0 = i * tile_w;
                t.ya = j * tile_h;
                t.yb = std::min(ny, (j + 1) * tile_h);
                tiles.push_back(t);
                std::vector<int>& w = wait[j * tx + i];
                std::sort(w.begin(), w.end());
                w.erase(std::unique(w.begin(), w.end()), w.end());
                if ((int)w.size() > lbm::BATCH_NEIGHBOURS)
                    return b->fail(LBM_ERR_ARG, "tiling too fine for a case: a tile would depend on more than 32 others");
                for (int k = 0; k < lbm::BATCH_NEIGHBOURS; ++k)
                    nbr.push_back(k < (int)w.size() ? base + w[k] : -1);
            }
    }
    if ((long long)tiles.size() > b->tiles_cap) return b->fail(LBM_ERR_WORKSPACE, "tile table larger than the workspace");
    int per_sm = occ();
    cudaGetLastError();
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || sms <= 0) sms = 1;
    if (per_sm <= 0) return b->fail(LBM_ERR_CUDA, "batched kernel does not fit on an SM");
    cudaError_t e = cudaMemcpyAsync(b->d_tiles(), tiles.data(), tiles.size() * sizeof(lbm::BatchTile),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_nbr(), nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the vectors are pageable
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_set_tiling", e);
    b->drop_graph();
    b->tile_w = tile_w;
    b->tile_h = tile_h;
    b->ntiles = (int)tiles.size();
    b->grid = (int)std::min<long long>(b->ntiles, (long long)per_sm * sms);
    b->launch = launch;
    e = b->reset_counters();
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_set_tiling", e);
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(lbm_handle* const* cases, int32_t ncases) {
    if (check_cases(cases, ncases, g_batch_error, sizeof(g_batch_error)) != LBM_OK) return 0;
    return batch_layout(ncases, max_tiles(cases, ncases)).total;
}

int lbm_batch_create(lbm_handle* const* cases, int32_t ncases, void* d_workspace, size_t workspace_bytes,
                     lbm_batch** out) {
    if (!out) { snprintf(g_batch_error, sizeof(g_batch_error), "out is NULL"); return LBM_ERR_ARG; }
    *out = nullptr;
    int rc = check_cases(cases, ncases, g_batch_error, sizeof(g_batch_error));
    if (rc != LBM_OK) return rc;
    const long long cap = max_tiles(cases, ncases);
    const BatchLayout L = batch_layout(ncases, cap);
    if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % BALIGN != 0 || workspace_bytes < L.total) {
        snprintf(g_batch_error, sizeof(g_batch_error),
                 "workspace must be a %zu-byte aligned device buffer of >= %zu bytes", BALIGN, L.total);
        return LBM_ERR_WORKSPACE;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) { snprintf(g_batch_error, sizeof(g_batch_error), "out of host memory"); return LBM_ERR_ARG; }
    b->cases.assign(cases, cases + ncases);
    b->device = cases[0]->device;
    b->q = cases[0]->p.scalar_q;
    b->stream = cases[0]->stream;
    b->ws = static_cast<uint8_t*>(d_workspace);
    b->L = L;
    b->tiles_cap = cap;
    lbm::detail::DeviceGuard dg(b->device);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&b->h_cases), (size_t)ncases * sizeof(lbm::BatchCase));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cases_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = b->make_side_streams();
    rc = e == cudaSuccess ? build_tiling(b, 128, 16) : b->fail(LBM_ERR_CUDA, "lbm_batch_create: staging", e);
    if (rc != LBM_OK) {
        snprintf(g_batch_error, sizeof(g_batch_error), "%s", b->err);
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch* b, int32_t tile_w, int32_t tile_h) {
    if (!b) return LBM_ERR_ARG;
    lbm::detail::DeviceGuard dg(b->device);
    return build_tiling(b, tile_w, tile_h);
}

int lbm_batch_tiling(const lbm_batch* b, int32_t* tile_w, int32_t* tile_h, int32_t* ntiles, int32_t* grid) {
    if (!b) return LBM_ERR_ARG;
    if (tile_w) *tile_w = b->tile_w;
    if (tile_h) *tile_h = b->tile_h;
    if (ntiles) *ntiles = b->ntiles;
    if (grid) *grid = b->grid;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    const lbm::NvtxRange range("lbm_batch_step");
    if (!b) return LBM_ERR_ARG;
    if (nsteps < 0) return b->fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (b->failed) return b->fail(LBM_ERR_TIMEOUT, "an earlier batched launch gave up waiting; set the tiling again after re-initialising the cases");
    if (nsteps == 0) return LBM_OK;
    lbm::detail::DeviceGuard dg(b->device);
    cudaError_t e = b->resync_cases();
    int64_t left = nsteps;
    const int G = lbm::detail::GRAPH_STEPS;
    if (e == cudaSuccess && left >= G) {
        if (!b->graph_tried) b->try_graph();
        while (e == cudaSuccess && left >= G) {
            e = b->graph ? cudaGraphLaunch(b->graph, b->stream) : b->launch_steps(G);
            left -= G;
        }
    }
    while (e == cudaSuccess && left > 0) {
        const int n = (int)std::min<int64_t>(left, 1 << 20);
        e = b->launch_steps(n);
        left -= n;
    }
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_step", e);
    b->steps += nsteps;
    for (lbm_handle* h : b->cases) {
        h->t += nsteps;
        h->cur = (h->cur + (int)(nsteps & 1)) & 1;
    }
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    lbm::detail::DeviceGuard dg(b->device);
    unsigned st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, b->d_status(), sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_sync", e);
    if (st != 0u) {
        b->failed = true;
        return b->fail(LBM_ERR_TIMEOUT, "a batched launch gave up waiting for a neighbouring tile");
    }
    for (size_t i = 0; i < b->cases.size(); ++i) {
        const int rc = lbm_sync(b->cases[i]);
        if (rc != LBM_OK) {
            snprintf(b->err, sizeof(b->err), "case %zu: %.400s", i, b->cases[i]->err);
            return rc;
        }
    }
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int32_t steps_per_trial, double* table, int32_t table_rows,
                       int32_t* rows_written) {
    if (!b) return LBM_ERR_ARG;
    if (steps_per_trial < 1) return b->fail(LBM_ERR_ARG, "steps_per_trial must be >= 1");
    lbm::detail::DeviceGuard dg(b->device);
    static const int widths[] = {32, 64, 128};
    static const int heights[] = {8, 16, 32, 64};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return b->fail(LBM_ERR_CUDA, "lbm_batch_autotune: events");
    }
    int best_w = b->tile_w, best_h = b->tile_h, rows = 0, rc = LBM_OK;
    double best = -1.0;
    for (int w : widths) {
        for (int hgt : heights) {
            rc = build_tiling(b, w, hgt);
            if (rc != LBM_OK) break;
            rc = lbm_batch_step(b, 2);  // first-touch of the new tables
            cudaError_t e = rc == LBM_OK ? cudaEventRecord(e0, b->stream) : cudaErrorUnknown;
            if (e == cudaSuccess) e = b->launch_steps(steps_per_trial);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { rc = rc != LBM_OK ? rc : b->fail(LBM_ERR_CUDA, "lbm_batch_autotune", e); break; }
            b->steps += steps_per_trial;
            for (lbm_handle* h : b->cases) {
                h->t += steps_per_trial;
                h->cur = (h->cur + (steps_per_trial & 1)) & 1;
            }
            rc = lbm_batch_sync(b);
            if (rc != LBM_OK) break;
            const double per_step = ms / steps_per_trial;
            if (table && rows < table_rows) {
                table[5 * rows + 0] = w;
                table[5 * rows + 1] = hgt;
                table[5 * rows + 2] = per_step;
                table[5 * rows + 3] = b->ntiles;
                table[5 * rows + 4] = b->grid;
                ++rows;
            }
            if (best < 0.0 || per_step < best) { best = per_step; best_w = w; best_h = hgt; }
        }
        if (rc != LBM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rows_written) *rows_written = rows;
    if (rc != LBM_OK) return rc;
    return build_tiling(b, best_w, best_h);
}

int lbm_batch_set_wait_limit(lbm_batch* b, int64_t spin_limit, int32_t hold_tile) {
    if (!b) return LBM_ERR_ARG;
    if (spin_limit < 1) return b->fail(LBM_ERR_ARG, "spin_limit must be >= 1");
    if (hold_tile < -1 || hold_tile >= b->ntiles) return b->fail(LBM_ERR_ARG, "hold_tile out of range");
    b->spin_limit = spin_limit;
    b->hold_tile = hold_tile;
    b->drop_graph();
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    lbm::detail::DeviceGuard dg(b->device);
    b->drop_graph();
    if (b->cases_ev) {
        if (b->cases_ev_live) cudaEventSynchronize(b->cases_ev);
        cudaEventDestroy(b->cases_ev);
    }
    if (b->h_cases) cudaFreeHost(b->h_cases);
    b->free_side_streams();  // work still queued on them completes first
    delete b;
}

int lbm_batch_init_macros(lbm_batch* b, const double* macros, int32_t on_device) {
    const lbm::NvtxRange range("lbm_batch_init_macros");
    if (!b) return LBM_ERR_ARG;
    if (!macros) return b->fail(LBM_ERR_ARG, "macros is NULL");
    lbm::detail::DeviceGuard dg(b->device);
    if (!on_device) {
        // host fields: each case stages its own copy (pageable memory), in turn
        size_t off = 0;
        for (size_t i = 0; i < b->cases.size(); ++i) {
            lbm_handle* h = b->cases[i];
            const size_t n = (size_t)h->p.nx * h->p.ny;
            const double* m = macros + off;
            const int rc = lbm_init_macros(h, m, m + n, m + 2 * n, m + 3 * n, m + 4 * n, m + 5 * n, 0);
            if (rc != LBM_OK) {
                snprintf(b->err, sizeof(b->err), "case %zu: %.400s", i, h->err);
                return rc;
            }
            off += 6 * n;
        }
        return LBM_OK;
    }
    std::vector<size_t> off(b->cases.size());
    for (size_t i = 0, o = 0; i < b->cases.size(); ++i) {
        off[i] = o;
        o += 6 * (size_t)b->cases[i]->p.nx * b->cases[i]->p.ny;
    }
    const cudaError_t e = b->fan_out([&](size_t i, cudaStream_t s) {
        lbm_handle* h = b->cases[i];
        const size_t n = (size_t)h->p.nx * h->p.ny;
        const double* m = macros + off[i];
        return h->init_on(lbm::InitFields{m, m + n, m + 2 * n, m + 3 * n, m + 4 * n, m + 5 * n}, s);
    });
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_init_macros", e);
    for (lbm_handle* h : b->cases) h->restarted();
    return LBM_OK;
}

int lbm_batch_get_fields(lbm_batch* b, uint32_t mask, void* out, int32_t out_on_device, int32_t out_dtype) {
    const lbm::NvtxRange range("lbm_batch_get_fields");
    if (!b) return LBM_ERR_ARG;
    mask &= LBM_FIELD_ALL;
    if (!mask || !out) return b->fail(LBM_ERR_ARG, "empty field mask or NULL output");
    if (out_dtype != LBM_OUT_F64 && out_dtype != LBM_OUT_F32) return b->fail(LBM_ERR_ARG, "out_dtype must be LBM_OUT_F64 or LBM_OUT_F32");
    lbm::detail::DeviceGuard dg(b->device);
    const size_t es = out_dtype == LBM_OUT_F64 ? sizeof(double) : sizeof(float);
    int k = 0;
    for (uint32_t m = mask; m; m &= m - 1) ++k;
    std::vector<size_t> off(b->cases.size());
    for (size_t i = 0, o = 0; i < b->cases.size(); ++i) {
        off[i] = o;
        o += (size_t)k * b->cases[i]->p.nx * b->cases[i]->p.ny;
    }
    uint8_t* base = static_cast<uint8_t*>(out);
    if (!out_on_device) {
        for (size_t i = 0; i < b->cases.size(); ++i) {
            lbm_handle* h = b->cases[i];
            const int rc = lbm_get_fields(h, mask, base + off[i] * es, 0, out_dtype);
            if (rc != LBM_OK) {
                snprintf(b->err, sizeof(b->err), "case %zu: %.400s", i, h->err);
                return rc;
            }
        }
        return LBM_OK;
    }
    const cudaError_t e = b->fan_out([&](size_t i, cudaStream_t s) {
        lbm_handle* h = b->cases[i];
        return h->fields(h->cur, mask, base + off[i] * es, out_dtype == LBM_OUT_F64, s);
    });
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_get_fields", e);
    return LBM_OK;
}

size_t lbm_batch_state_bytes(const lbm_batch* b) {
    if (!b) return 0;
    size_t n = 0;
    for (const lbm_handle* h : b->cases) n += h->state_bytes();
    return n;
}

static int batch_state_copy(lbm_batch* b, void* buf, size_t bytes, int32_t on_device, bool get) {
    if (!b) return LBM_ERR_ARG;
    if (!buf || bytes < lbm_batch_state_bytes(b)) return b->fail(LBM_ERR_ARG, "state buffer NULL or smaller than lbm_batch_state_bytes()");
    lbm::detail::DeviceGuard dg(b->device);
    std::vector<size_t> off(b->cases.size());
    for (size_t i = 0, o = 0; i < b->cases.size(); ++i) {
        off[i] = o;
        o += b->cases[i]->state_bytes();
    }
    uint8_t* base = static_cast<uint8_t*>(buf);
    if (!on_device) {
        for (size_t i = 0; i < b->cases.size(); ++i) {
            lbm_handle* h = b->cases[i];
            const size_t n = h->state_bytes();
            const int rc = get ? lbm_get_state(h, base + off[i], n, 0) : lbm_set_state(h, base + off[i], n, 0);
            if (rc != LBM_OK) {
                snprintf(b->err, sizeof(b->err), "case %zu: %.400s", i, h->err);
                return rc;
            }
        }
        return LBM_OK;
    }
    const cudaError_t e = b->fan_out([&](size_t i, cudaStream_t s) {
        return b->cases[i]->copy_state(base + off[i], get, true, s);
    });
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, get ? "lbm_batch_get_state" : "lbm_batch_set_state", e);
    if (!get)
        for (lbm_handle* h : b->cases) h->restarted();
    return LBM_OK;
}

int lbm_batch_get_state(lbm_batch* b, void* buf, size_t bytes, int32_t on_device) {
    return batch_state_copy(b, buf, bytes, on_device, true);
}

int lbm_batch_set_state(lbm_batch* b, const void* buf, size_t bytes, int32_t on_device) {
    return batch_state_copy(b, const_cast<void*>(buf), bytes, on_device, false);
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_batch_error; }

}  // extern "C"
