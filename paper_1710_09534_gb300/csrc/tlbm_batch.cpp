// C ABI of batched execution (include/tlbm.h, "Batches"): membership,
// device descriptors and work lists, the captured CUDA graph of a step pair,
// and the tile-shape / work-split tuner.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tlbm.h"
#include "tlbm_batch.cuh"
#include "tlbm_internal.h"

namespace {

constexpr int64_t kAlign = 256;
int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int err(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return tlb::set_error(code, buf);
}

#define B_CUDA(call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return err(TLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct BatchLayout {
    int64_t desc = 0, tiles = 0, walls = 0, ctr = 0, total = 0;
};

BatchLayout batch_layout(int max_lattices, int64_t max_tiles, int64_t max_wall)
{
    BatchLayout b;
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const int64_t desc_max = (int64_t)std::max(sizeof(tlb::LatDesc<double>), sizeof(tlb::LatDesc<float>));
    b.desc = take(desc_max * max_lattices);
    b.tiles = take((int64_t)sizeof(tlb::TileItem) * max_tiles);
    b.walls = take((int64_t)sizeof(tlb::WallItem) * max_wall);
    b.ctr = take(sizeof(tlb::BatchCounters));
    b.total = off;
    return b;
}

}  // namespace

struct tlb_batch {
    int precision = 0, device = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    BatchLayout lay;
    int max_lattices = 0;
    int64_t max_tiles = 0, max_wall = 0;
    const tlb::Ops* ops = nullptr;
    std::vector<tlb_lattice*> members;
    std::vector<int> member_cur;  // each member's buffer parity when the descriptors were built
    int variant = 1;              // 0: 64-thread tiles, 1: 128-thread tiles
    int rows_small = 16, rows_large = 16, small_ny = 128;
    bool dirty = true;
    int64_t n_tiles = 0, n_wall = 0;
    int grid_interior = 0, grid_wall = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_variant = -1;
    const tlb::Ops* graph_ops = nullptr;
    // the near-wall loop of a step runs on `side`, concurrently with the
    // interior tile queue (disjoint writes, one state read), between `fork`
    // and `join` (captured into the graph like the launches)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

int rows_for(const tlb_batch* B, const tlb_lattice* L) { return L->ny <= B->small_ny ? B->rows_small : B->rows_large; }

int64_t tiles_of(int variant, int rows, int nx, int ny)
{
    const int tx = (variant == 0 ? 64 : 128) - 4;
    return (int64_t)((nx + tx - 1) / tx) * ((ny + rows - 1) / rows);
}

// Device descriptors, tile list (members largest first, each member's tiles
// contiguous so that neighbouring segments run together) and wall list.
int rebuild(tlb_batch* B)
{
    // one collision model per batch: the members' launch tables must agree
    if (!B->members.empty()) {
        for (const tlb_lattice* L : B->members)
            if (L->ops != B->members[0]->ops)
                return err(TLB_EINVAL, "batch members use different collision models (BGK and MRT)");
        B->ops = B->members[0]->ops;
    }
    const size_t ds = B->ops->desc_size;
    std::vector<char> descs(ds * B->members.size());
    std::vector<int> order(B->members.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return B->members[a]->n() > B->members[b]->n(); });
    std::vector<tlb::TileItem> tiles;
    std::vector<tlb::WallItem> walls;
    const int tx = (B->variant == 0 ? 64 : 128) - 4;
    for (size_t i = 0; i < B->members.size(); i++) {
        tlb_lattice* L = B->members[i];
        B->ops->fill_desc(descs.data() + ds * i, L->bufA(), L->bufB(), L->cu(), L->dcls(), L->geo, L->prm,
                          rows_for(B, L));
        B->member_cur[i] = L->cur;
    }
    for (int i : order) {
        tlb_lattice* L = B->members[i];
        const int rows = rows_for(B, L);
        const int nbx = (L->nx + tx - 1) / tx, nby = (L->ny + rows - 1) / rows;
        for (int by = 0; by < nby; by++)
            for (int bx = 0; bx < nbx; bx++) tiles.push_back({i, bx, by});
        for (uint32_t p : L->hlist) walls.push_back({i, p});
    }
    if ((int64_t)tiles.size() > B->max_tiles || (int64_t)walls.size() > B->max_wall)
        return err(TLB_ENOMEM, "batch needs %zu tiles and %zu wall nodes; capacity %lld and %lld", tiles.size(),
                   walls.size(), (long long)B->max_tiles, (long long)B->max_wall);
    tlb::BatchCounters c{(int)tiles.size(), (int)walls.size(), {0, 0}};
    if (!descs.empty())
        B_CUDA(cudaMemcpyAsync(B->ws + B->lay.desc, descs.data(), descs.size(), cudaMemcpyHostToDevice, B->stream));
    if (!tiles.empty())
        B_CUDA(cudaMemcpyAsync(B->ws + B->lay.tiles, tiles.data(), tiles.size() * sizeof(tlb::TileItem),
                               cudaMemcpyHostToDevice, B->stream));
    if (!walls.empty())
        B_CUDA(cudaMemcpyAsync(B->ws + B->lay.walls, walls.data(), walls.size() * sizeof(tlb::WallItem),
                               cudaMemcpyHostToDevice, B->stream));
    B_CUDA(cudaMemcpyAsync(B->ws + B->lay.ctr, &c, sizeof c, cudaMemcpyHostToDevice, B->stream));
    B_CUDA(cudaStreamSynchronize(B->stream));
    B->n_tiles = (int64_t)tiles.size();
    B->n_wall = (int64_t)walls.size();
    int sms = 0;
    B_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device));
    const int per_sm = std::max(1, B->ops->batch_blocks_per_sm(B->variant));
    B->grid_interior = sms * per_sm;
    B->grid_wall = 2 * sms;
    B->dirty = false;
    return TLB_OK;
}

int launch_step(tlb_batch* B, int parity)
{
    B_CUDA(cudaEventRecord(B->fork, B->stream));
    B_CUDA(cudaStreamWaitEvent(B->side, B->fork, 0));
    B_CUDA(B->ops->batch_step(B->ws + B->lay.desc, B->ws + B->lay.tiles, B->ws + B->lay.walls, B->ws + B->lay.ctr,
                              parity, B->variant, B->grid_interior, B->grid_wall, B->stream, B->side));
    B_CUDA(cudaEventRecord(B->join, B->side));
    B_CUDA(cudaStreamWaitEvent(B->stream, B->join, 0));
    return TLB_OK;
}

// Graph of one even and one odd step (valid for any membership: the counts
// and descriptors live in device memory).
int ensure_graph(tlb_batch* B)
{
    if (B->graph && B->graph_variant == B->variant && B->graph_ops == B->ops) return TLB_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    B_CUDA(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_step(B, 0);
    if (rc == TLB_OK) rc = launch_step(B, 1);
    const cudaError_t e = cudaStreamEndCapture(B->stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return err(TLB_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return err(TLB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ei));
    B->graph_variant = B->variant;
    B->graph_ops = B->ops;
    return TLB_OK;
}

int check_batch(tlb_batch* B)
{
    if (!B) return err(TLB_EINVAL, "null batch handle");
    B_CUDA(cudaSetDevice(B->device));
    return TLB_OK;
}

int advance(tlb_batch* B, int64_t n, bool use_graph)
{
    for (size_t i = 0; i < B->members.size(); i++) {
        tlb_lattice* L = B->members[i];
        if (!L->have_params || !L->have_fields) return err(TLB_ESTATE, "member %zu has no state", i);
        if (L->cur != B->member_cur[i]) B->dirty = true;
    }
    int rc;
    if (B->dirty && (rc = rebuild(B))) return rc;
    if (B->members.empty() || n == 0) return TLB_OK;
    if (use_graph && n >= 2) {
        if ((rc = ensure_graph(B))) return rc;
        for (int64_t s = 0; s + 1 < n; s += 2) B_CUDA(cudaGraphLaunch(B->graph, B->stream));
    } else {
        for (int64_t s = 0; s + 1 < n; s += 2) {
            if ((rc = launch_step(B, 0)) || (rc = launch_step(B, 1))) return rc;
        }
    }
    if (n & 1) {
        if ((rc = launch_step(B, 0))) return rc;
        for (size_t i = 0; i < B->members.size(); i++) B->members[i]->cur ^= 1;
        B->dirty = true;
    }
    return TLB_OK;
}

// Bytes of one member's c_i u planes (Eq. 19), the only state a step
// updates in place.
int64_t cu_bytes(const tlb_lattice* L) { return 4 * L->lay.plane * (int64_t)tlb::cu_elem_for(L->precision); }

int64_t tune_scratch_bytes(const tlb_batch* B)
{
    int64_t total = 0;
    for (const tlb_lattice* L : B->members) total += align_up(cu_bytes(L));
    return total;
}

// n trial steps that leave every member's state as it was, apart from the
// c_i u planes: each reads the members' current buffer and writes the spare
// one (the step parity is never flipped), so the current distributions are
// untouched; the caller saves and restores the c_i u planes around them.
int trial_steps(tlb_batch* B, int64_t n)
{
    int rc;
    if (B->dirty && (rc = rebuild(B))) return rc;
    for (int64_t s = 0; s < n; s++)
        if ((rc = launch_step(B, 0))) return rc;
    return TLB_OK;
}

// Copy every member's c_i u planes to (save = true) or from the scratch.
int copy_cu(tlb_batch* B, char* scratch, bool save)
{
    int64_t off = 0;
    for (tlb_lattice* L : B->members) {
        const int64_t nb = cu_bytes(L);
        char* keep = scratch + off;
        B_CUDA(cudaMemcpyAsync(save ? keep : (char*)L->cu(), save ? (const char*)L->cu() : keep, (size_t)nb,
                               cudaMemcpyDeviceToDevice, B->stream));
        off += align_up(nb);
    }
    return TLB_OK;
}

}  // namespace

namespace tlb {
void batch_member_changed(tlb_batch* B)
{
    if (B) B->dirty = true;
}

int batch_sync(tlb_batch* B)
{
    if (!B) return TLB_OK;
    const cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return err(TLB_ECUDA, "batch stream: %s", cudaGetErrorString(e));
    return TLB_OK;
}
}  // namespace tlb

extern "C" {

int64_t tlb_batch_workspace_bytes(int max_lattices, int64_t max_tiles, int64_t max_wall_nodes)
{
    if (max_lattices < 1 || max_tiles < 1 || max_wall_nodes < 0) return err(TLB_EINVAL, "bad batch capacity");
    tlb::clear_error();
    return batch_layout(max_lattices, max_tiles, max_wall_nodes).total;
}

int64_t tlb_batch_tiles_needed(int nx, int ny)
{
    if (nx < 3 || ny < 3) return err(TLB_EINVAL, "lattice size %dx%d out of range", nx, ny);
    tlb::clear_error();
    // the smallest tiles the tuner may pick: 64-thread strips, 8-row segments
    return tiles_of(0, 8, nx, ny);
}

int tlb_batch_create(int precision, int max_lattices, int64_t max_tiles, int64_t max_wall_nodes,
                     void* dev_workspace, int64_t ws_bytes, void* cuda_stream, tlb_batch** out)
{
    if (!out) return err(TLB_EINVAL, "out is null");
    *out = nullptr;
    if (precision < TLB_FP64 || precision > TLB_BF16) return err(TLB_EINVAL, "unknown precision %d", precision);
    if (max_lattices < 1 || max_tiles < 1 || max_wall_nodes < 0) return err(TLB_EINVAL, "bad batch capacity");
    if (!cuda_stream) return err(TLB_EINVAL, "a batch needs a non-default stream (it is graph-captured)");
    const BatchLayout lay = batch_layout(max_lattices, max_tiles, max_wall_nodes);
    if (!dev_workspace || ((uintptr_t)dev_workspace) % kAlign) return err(TLB_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total) return err(TLB_ENOMEM, "batch workspace has %lld bytes, needs %lld", (long long)ws_bytes, (long long)lay.total);
    auto* B = new tlb_batch;
    B->precision = precision;
    B->stream = (cudaStream_t)cuda_stream;
    B->ws = (char*)dev_workspace;
    B->lay = lay;
    B->max_lattices = max_lattices;
    B->max_tiles = max_tiles;
    B->max_wall = max_wall_nodes;
    B->ops = &tlb::ops_for(precision, false);
    if (cudaGetDevice(&B->device) != cudaSuccess) {
        delete B;
        return err(TLB_ECUDA, "no current device");
    }
    cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (B->fork) cudaEventDestroy(B->fork);
        if (B->join) cudaEventDestroy(B->join);
        delete B;
        return err(TLB_ECUDA, "batch set-up failed: %s", cudaGetErrorString(e));
    }
    *out = B;
    return tlb::clear_error();
}

int tlb_batch_add(tlb_batch* B, tlb_lattice* L)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (!L) return err(TLB_EINVAL, "null lattice");
    if (L->batch) return err(TLB_EINVAL, "lattice already belongs to a batch");
    if (L->precision != B->precision) return err(TLB_EINVAL, "lattice precision differs from the batch's");
    if (L->lay.inplace) return err(TLB_EINVAL, "in-place lattices are stepped alone, not in a batch");
    if (L->device != B->device) return err(TLB_EINVAL, "lattice lives on another device");
    if ((int)B->members.size() >= B->max_lattices) return err(TLB_ENOMEM, "batch is full (%d lattices)", B->max_lattices);
    // work queued on the lattice's own stream must be done before the batch stream touches it
    B_CUDA(cudaStreamSynchronize(L->stream));
    B->members.push_back(L);
    B->member_cur.push_back(-1);
    L->batch = B;
    B->dirty = true;
    return tlb::clear_error();
}

int tlb_batch_remove(tlb_batch* B, tlb_lattice* L)
{
    int rc = check_batch(B);
    if (rc) return rc;
    auto it = std::find(B->members.begin(), B->members.end(), L);
    if (it == B->members.end()) return err(TLB_EINVAL, "lattice is not in this batch");
    // the batch stream may still be stepping it
    B_CUDA(cudaStreamSynchronize(B->stream));
    const size_t i = (size_t)(it - B->members.begin());
    B->members.erase(it);
    B->member_cur.erase(B->member_cur.begin() + (long)i);
    L->batch = nullptr;
    B->dirty = true;
    return tlb::clear_error();
}

int tlb_batch_size(tlb_batch* B)
{
    if (!B) return err(TLB_EINVAL, "null batch handle");
    return (int)B->members.size();
}

int tlb_batch_step(tlb_batch* B, int64_t n)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (n < 0) return err(TLB_EINVAL, "negative step count");
    if ((rc = advance(B, n, true))) return rc;
    return tlb::clear_error();
}

int tlb_batch_config(tlb_batch* B, int threads, int rows_small, int rows_large, int small_ny)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if ((threads != 64 && threads != 128) || rows_small < 2 || rows_large < 2 || small_ny < 0)
        return err(TLB_EINVAL, "threads must be 64 or 128 and rows >= 2");
    B->variant = threads == 64 ? 0 : 1;
    B->rows_small = rows_small;
    B->rows_large = rows_large;
    B->small_ny = small_ny;
    B->dirty = true;
    return tlb::clear_error();
}

int64_t tlb_batch_tune_scratch_bytes(tlb_batch* B)
{
    if (!B) return err(TLB_EINVAL, "null batch handle");
    tlb::clear_error();
    return tune_scratch_bytes(B);
}

int tlb_batch_tune(tlb_batch* B, int trial_steps_n, void* dev_scratch, int64_t scratch_bytes, int out_config[4],
                   double* out_ms_per_step)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (trial_steps_n < 1) return err(TLB_EINVAL, "trial_steps must be >= 1");
    if (B->members.empty()) return err(TLB_ESTATE, "empty batch");
    for (size_t i = 0; i < B->members.size(); i++) {
        const tlb_lattice* L = B->members[i];
        if (!L->have_params || !L->have_fields) return err(TLB_ESTATE, "member %zu has no state", i);
    }
    const int64_t need = tune_scratch_bytes(B);
    if (!dev_scratch || ((uintptr_t)dev_scratch) % kAlign) return err(TLB_EINVAL, "scratch must be 256-byte aligned device memory");
    if (scratch_bytes < need)
        return err(TLB_ENOMEM, "tuning scratch has %lld bytes, needs %lld", (long long)scratch_bytes, (long long)need);
    B_CUDA(cudaStreamSynchronize(B->stream));
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return err(TLB_ECUDA, "cudaEventCreate failed");
    }
    const int shapes[][3] = {{128, 16, 16}, {128, 8, 16}, {128, 8, 32}, {128, 16, 32},
                             {64, 8, 16}, {64, 16, 16}, {64, 8, 32}, {64, 16, 32}};
    const int saved[4] = {B->variant, B->rows_small, B->rows_large, B->small_ny};
    double best = 1e30;
    int best_i = 0;
    rc = copy_cu(B, (char*)dev_scratch, true);
    for (int i = 0; rc == TLB_OK && i < (int)(sizeof shapes / sizeof shapes[0]); i++) {
        B->variant = shapes[i][0] == 64 ? 0 : 1;
        B->rows_small = shapes[i][1];
        B->rows_large = shapes[i][2];
        B->small_ny = 128;
        B->dirty = true;
        if ((rc = trial_steps(B, 2))) break;  // warm-up (also rebuilds the lists)
        cudaError_t ce = cudaEventRecord(e0, B->stream);
        if (ce == cudaSuccess && (rc = trial_steps(B, trial_steps_n)) == TLB_OK) ce = cudaEventRecord(e1, B->stream);
        if (rc) break;
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
            rc = err(TLB_ECUDA, "tuner timing failed: %s", cudaGetErrorString(ce));
            break;
        }
        if (ms / trial_steps_n < best) {
            best = ms / trial_steps_n;
            best_i = i;
        }
    }
    // put back the c_i u planes the trial steps overwrote (the distributions
    // of the current buffer were only read)
    const int rc_restore = copy_cu(B, (char*)dev_scratch, false);
    const cudaError_t es = cudaStreamSynchronize(B->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->dirty = true;
    if (rc || rc_restore) {
        B->variant = saved[0];
        B->rows_small = saved[1];
        B->rows_large = saved[2];
        B->small_ny = saved[3];
        return rc ? rc : rc_restore;
    }
    if (es != cudaSuccess) return err(TLB_ECUDA, "batch stream: %s", cudaGetErrorString(es));
    B->variant = shapes[best_i][0] == 64 ? 0 : 1;
    B->rows_small = shapes[best_i][1];
    B->rows_large = shapes[best_i][2];
    if (out_config) {
        out_config[0] = shapes[best_i][0];
        out_config[1] = shapes[best_i][1];
        out_config[2] = shapes[best_i][2];
        out_config[3] = B->small_ny;
    }
    if (out_ms_per_step) *out_ms_per_step = best;
    return tlb::clear_error();
}

void tlb_batch_destroy(tlb_batch* B)
{
    if (!B) return;
    cudaSetDevice(B->device);
    cudaStreamSynchronize(B->stream);
    for (tlb_lattice* L : B->members) L->batch = nullptr;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaEventDestroy(B->fork);
    cudaEventDestroy(B->join);
    cudaStreamDestroy(B->side);
    delete B;
}

}  // extern "C"
