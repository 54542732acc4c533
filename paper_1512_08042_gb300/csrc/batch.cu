// Batched ensemble: independent channels (replicas), each with its own parameters, advanced
// by one launch per kernel for all of them per hybrid step. Each replica is an ordinary
// context in its own part of one caller-owned arena; after the replicas' arenas comes a table
// region with the per-replica kernel arguments of every ping-pong parity and the prefix sums
// that map a launch's units to replicas. The kernels are the single-context ones in their
// batch form (Launch with a table), so a replica advanced in a batch and the same channel
// advanced alone give the same results.
#include <cstring>
#include <new>
#include <vector>

#include "hyb_internal.cuh"

using hyb::BatchDev;
using hyb::Ctx;

struct hyb_batch {
    BatchDev dev;
    std::vector<hyb_ctx*> reps;
    char* arena = nullptr;
    cudaStream_t stream = nullptr;
    int cur_p = 0, cur_f = 0;
    // table region
    char* tab = nullptr;
    uint64_t off_dsmc[2] = {}, off_lbm[2] = {}, off_d2l[2][2] = {}, off_l2d[2][2] = {};
    uint64_t off_pre_cells = 0, off_pre_blocks = 0, off_pre_blocks4 = 0, off_pre_nodes = 0, off_pre_d2l = 0,
             off_pre_l2d = 0;
    // coupling lists of the tables and graphs
    const int32_t* nodes = nullptr;
    const int32_t* cells = nullptr;
    std::vector<int64_t> node_pre, cell_pre;
    bool lists_set = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int g_curf[2] = {0, 0};
    std::string err;
};

namespace {

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Offsets of the table region's parts, relative to its start; returns its size.
uint64_t table_layout(int n, int real_bytes, hyb_batch* b) {
    const uint64_t ds = hyb::dsmc_args_bytes(real_bytes), ls = hyb::lbm_args_bytes(real_bytes),
                   ms = hyb::map_args_bytes(real_bytes);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const uint64_t d0 = take(n * ds), d1 = take(n * ds);
    const uint64_t l0 = take(n * ls), l1 = take(n * ls);
    uint64_t md[2][2], ml[2][2];
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 2; ++f) {
            md[p][f] = take(n * ms);
            ml[p][f] = take(n * ms);
        }
    const uint64_t pc = take((n + 1) * 8), pb = take((n + 1) * 8), pb4 = take((n + 1) * 8),
                   pn = take((n + 1) * 8), pd = take((n + 1) * 8), pl = take((n + 1) * 8);
    if (b) {
        b->off_dsmc[0] = d0;
        b->off_dsmc[1] = d1;
        b->off_lbm[0] = l0;
        b->off_lbm[1] = l1;
        for (int p = 0; p < 2; ++p)
            for (int f = 0; f < 2; ++f) {
                b->off_d2l[p][f] = md[p][f];
                b->off_l2d[p][f] = ml[p][f];
            }
        b->off_pre_cells = pc;
        b->off_pre_blocks = pb;
        b->off_pre_blocks4 = pb4;
        b->off_pre_nodes = pn;
        b->off_pre_d2l = pd;
        b->off_pre_l2d = pl;
    }
    return off;
}

bool same_kind(const hyb_params* p, int n) {
    for (int r = 0; r < n; ++r)
        if (p[r].real_bytes != p[0].real_bytes || p[r].lattice != p[0].lattice ||
            p[r].lb_collision != p[0].lb_collision || p[r].kn_profile != 0 || p[r].ncz >= 2 ||
            p[r].ncy_global != 0)
            return false;
    return true;
}

hyb_status bcheck(hyb_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HYB_OK;
    b->err = what;
    b->err += ": ";
    b->err += cudaGetErrorString(e);
    return HYB_ECUDA;
}

void drop_graphs(hyb_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

// Uploads the DSMC2LB and LB2DSMC argument tables for the given coupling lists.
hyb_status set_lists(hyb_batch* b, const int32_t* nodes, const int64_t* node_pre, const int32_t* cells,
                     const int64_t* cell_pre) {
    const int n = b->dev.nrep;
    const int rb = b->dev.real_bytes;
    const uint64_t ms = hyb::map_args_bytes(rb);
    hyb_status s = bcheck(b, cudaStreamSynchronize(b->stream), "synchronize");  // tables in use
    if (s != HYB_OK) return s;
    std::vector<char> host(4 * n * ms);
    for (int kind = 0; kind < 2; ++kind) {
        const int32_t* list = kind == 0 ? nodes : cells;
        const int64_t* pre = kind == 0 ? node_pre : cell_pre;
        for (int p = 0; p < 2; ++p)
            for (int f = 0; f < 2; ++f) {
                for (int r = 0; r < n; ++r) {
                    const int64_t cnt = pre[r + 1] - pre[r];
                    hyb::map_args_fill(b->reps[r]->c, p, f, list ? list + pre[r] : nullptr, (int32_t)cnt,
                                       host.data() + (size_t)r * ms);
                }
                const uint64_t off = kind == 0 ? b->off_d2l[p][f] : b->off_l2d[p][f];
                s = bcheck(b, cudaMemcpy(b->tab + off, host.data(), n * ms, cudaMemcpyHostToDevice),
                           "upload mapping arguments");
                if (s != HYB_OK) return s;
            }
        s = bcheck(b, cudaMemcpy(b->tab + (kind == 0 ? b->off_pre_d2l : b->off_pre_l2d), pre, (n + 1) * 8,
                                 cudaMemcpyHostToDevice),
                   "upload list offsets");
        if (s != HYB_OK) return s;
    }
    b->dev.tot_d2l = node_pre[n];
    b->dev.tot_l2d = cell_pre[n];
    b->nodes = nodes;
    b->cells = cells;
    b->node_pre.assign(node_pre, node_pre + n + 1);
    b->cell_pre.assign(cell_pre, cell_pre + n + 1);
    b->lists_set = true;
    drop_graphs(b);
    return HYB_OK;
}

// One hybrid step of every replica, in the order of a single context's hybrid step.
hyb_status batch_step(hyb_batch* b, int cur_p, int cur_f) {
    BatchDev& d = b->dev;
    hyb_status s = bcheck(b, hyb::launch_batch_move(d, cur_p), "batch move");
    if (s != HYB_OK) return s;
    s = bcheck(b, hyb::launch_batch_collide(d, cur_p), "batch collide");
    if (s != HYB_OK) return s;
    const int np = cur_p ^ 1;
    if (d.tot_d2l > 0) {
        s = bcheck(b, hyb::launch_batch_d2l(d, np, cur_f), "batch map_dsmc_to_lbm");
        if (s != HYB_OK) return s;
    }
    s = bcheck(b, hyb::launch_batch_lbm(d, cur_f), "batch lbm");
    if (s != HYB_OK) return s;
    if (d.tot_l2d > 0) s = bcheck(b, hyb::launch_batch_l2d(d, np, cur_f ^ 1), "batch map_lbm_to_dsmc");
    return s;
}

void flip(hyb_batch* b) {
    b->cur_p ^= 1;
    b->cur_f ^= 1;
    for (hyb_ctx* h : b->reps) {
        h->c.cur_p ^= 1;
        h->c.cur_f ^= 1;
    }
}

bool in_lockstep(const hyb_batch* b) {
    for (const hyb_ctx* h : b->reps)
        if (h->c.cur_p != b->cur_p || h->c.cur_f != b->cur_f) return false;
    return true;
}

bool lists_match(const hyb_batch* b, const int32_t* nodes, const int64_t* node_pre, const int32_t* cells,
                 const int64_t* cell_pre) {
    if (!b->lists_set || b->nodes != nodes || b->cells != cells) return false;
    const int n = b->dev.nrep;
    return std::memcmp(b->node_pre.data(), node_pre, (n + 1) * 8) == 0 &&
           std::memcmp(b->cell_pre.data(), cell_pre, (n + 1) * 8) == 0;
}

}  // namespace

extern "C" {

hyb_status hyb_batch_layout(const hyb_params* p, int32_t n, uint64_t* offsets) {
    if (!p || n < 1 || !offsets || !same_kind(p, n)) return HYB_EINVAL;
    uint64_t off = 0;
    for (int r = 0; r < n; ++r) {
        hyb_layout L;
        if (hyb_layout_compute(&p[r], &L) != HYB_OK) return HYB_EINVAL;
        offsets[r] = off;
        off = align256(off + L.total_bytes);
    }
    offsets[n] = off;
    offsets[n + 1] = off + table_layout(n, p[0].real_bytes, nullptr);
    return HYB_OK;
}

hyb_status hyb_batch_init(const hyb_params* p, int32_t n, void* arena, uint64_t arena_bytes, void* stream,
                          hyb_batch** out) {
    if (!out || !p || n < 1 || !arena || ((uintptr_t)arena & 255u)) return HYB_EINVAL;
    *out = nullptr;
    std::vector<uint64_t> off(n + 2);
    if (hyb_batch_layout(p, n, off.data()) != HYB_OK) return HYB_EINVAL;
    if (arena_bytes < off[n + 1]) return HYB_ENOMEM;
    hyb_batch* b = new (std::nothrow) hyb_batch();
    if (!b) return HYB_ENOMEM;
    b->arena = (char*)arena;
    b->stream = (cudaStream_t)stream;
    for (int r = 0; r < n; ++r) {
        hyb_layout L;
        hyb_layout_compute(&p[r], &L);
        hyb_ctx* h = nullptr;
        const hyb_status s = dsmc_init(&p[r], b->arena + off[r], L.total_bytes, stream, &h);
        if (s != HYB_OK) {
            hyb_batch_destroy(b);
            return s;
        }
        b->reps.push_back(h);
    }
    BatchDev& d = b->dev;
    d.nrep = n;
    d.real_bytes = p[0].real_bytes;
    d.lattice = p[0].lattice;
    d.lb_collision = p[0].lb_collision;
    d.stream = b->stream;
    d.num_sms = b->reps[0]->c.num_sms;
    b->cur_p = b->reps[0]->c.cur_p;
    b->cur_f = b->reps[0]->c.cur_f;
    b->tab = b->arena + off[n];
    table_layout(n, d.real_bytes, b);
    // prefix sums of the units and the DSMC and LB argument tables of both parities
    std::vector<int64_t> pc(n + 1, 0), pb(n + 1, 0), pb4(n + 1, 0), pn(n + 1, 0);
    for (int r = 0; r < n; ++r) {
        const Ctx& c = b->reps[r]->c;
        pc[r + 1] = pc[r] + c.d.ncells;
        pb[r + 1] = pb[r] + (c.d.ncells + 31) / 32;  // collide blocks of 32 cells
        pb4[r + 1] = pb4[r] + (c.d.ncells + 15) / 16;  // and of 16
        pn[r + 1] = pn[r] + c.d.nnodes;
        const uint32_t pool = hyb::collide_pool(c, 8), pool4 = hyb::collide_pool(c, 4);
        if (pool > d.pool) d.pool = pool;
        if (pool4 > d.pool4) d.pool4 = pool4;
        if ((uint32_t)c.d.bin > d.maxbin) d.maxbin = (uint32_t)c.d.bin;
    }
    d.tot_cells = pc[n];
    d.tot_blocks = pb[n];
    d.tot_blocks4 = pb4[n];
    d.tot_nodes = pn[n];
    const uint64_t ds = hyb::dsmc_args_bytes(d.real_bytes), ls = hyb::lbm_args_bytes(d.real_bytes);
    std::vector<char> host(n * (ds > ls ? ds : ls));
    hyb_status s = HYB_OK;
    for (int h = 0; h < 2 && s == HYB_OK; ++h) {
        for (int r = 0; r < n; ++r) hyb::dsmc_args_fill(b->reps[r]->c, h, host.data() + (size_t)r * ds);
        s = bcheck(b, cudaMemcpy(b->tab + b->off_dsmc[h], host.data(), n * ds, cudaMemcpyHostToDevice),
                   "upload DSMC arguments");
        if (s != HYB_OK) break;
        for (int r = 0; r < n; ++r) hyb::lbm_args_fill(b->reps[r]->c, h, host.data() + (size_t)r * ls);
        s = bcheck(b, cudaMemcpy(b->tab + b->off_lbm[h], host.data(), n * ls, cudaMemcpyHostToDevice),
                   "upload LB arguments");
    }
    if (s == HYB_OK) s = bcheck(b, cudaMemcpy(b->tab + b->off_pre_cells, pc.data(), (n + 1) * 8, cudaMemcpyHostToDevice), "upload offsets");
    if (s == HYB_OK) s = bcheck(b, cudaMemcpy(b->tab + b->off_pre_blocks, pb.data(), (n + 1) * 8, cudaMemcpyHostToDevice), "upload offsets");
    if (s == HYB_OK) s = bcheck(b, cudaMemcpy(b->tab + b->off_pre_blocks4, pb4.data(), (n + 1) * 8, cudaMemcpyHostToDevice), "upload offsets");
    if (s == HYB_OK) s = bcheck(b, cudaMemcpy(b->tab + b->off_pre_nodes, pn.data(), (n + 1) * 8, cudaMemcpyHostToDevice), "upload offsets");
    if (s != HYB_OK) {
        hyb_batch_destroy(b);
        return s;
    }
    for (int h = 0; h < 2; ++h) {
        d.dsmc[h] = b->tab + b->off_dsmc[h];
        d.lbm[h] = b->tab + b->off_lbm[h];
        for (int f = 0; f < 2; ++f) {
            d.d2l[h][f] = b->tab + b->off_d2l[h][f];
            d.l2d[h][f] = b->tab + b->off_l2d[h][f];
        }
    }
    d.pre_cells = (const int64_t*)(b->tab + b->off_pre_cells);
    d.pre_blocks = (const int64_t*)(b->tab + b->off_pre_blocks);
    d.pre_blocks4 = (const int64_t*)(b->tab + b->off_pre_blocks4);
    d.pre_nodes = (const int64_t*)(b->tab + b->off_pre_nodes);
    d.pre_d2l = (const int64_t*)(b->tab + b->off_pre_d2l);
    d.pre_l2d = (const int64_t*)(b->tab + b->off_pre_l2d);
    *out = b;
    return HYB_OK;
}

hyb_status hyb_batch_replica(hyb_batch* b, int32_t r, hyb_ctx** out) {
    if (!b || !out || r < 0 || r >= (int32_t)b->reps.size()) return HYB_EINVAL;
    *out = b->reps[r];
    return HYB_OK;
}

hyb_status hyb_batch_hybrid_step(hyb_batch* b, const int32_t* dev_nodes, const int64_t* node_pre,
                                 const int32_t* dev_cells, const int64_t* cell_pre, int32_t nsteps,
                                 int32_t use_graph) {
    if (!b || nsteps < 0 || !node_pre || !cell_pre) return HYB_EINVAL;
    const int n = b->dev.nrep;
    if (node_pre[0] != 0 || cell_pre[0] != 0) return HYB_EINVAL;
    for (int r = 0; r < n; ++r) {
        const Ctx& c = b->reps[r]->c;
        const int64_t nn = node_pre[r + 1] - node_pre[r], nc = cell_pre[r + 1] - cell_pre[r];
        if (nn < 0 || nc < 0 || nn > c.d.nnodes || nc > c.d.ncells) return HYB_EINVAL;
    }
    if ((node_pre[n] > 0 && !dev_nodes) || (cell_pre[n] > 0 && !dev_cells)) return HYB_EINVAL;
    if (!in_lockstep(b)) {
        b->err = "a replica was stepped on its own: the batch is out of lockstep";
        return HYB_ESTATE;
    }
    if (!lists_match(b, dev_nodes, node_pre, dev_cells, cell_pre)) {
        const hyb_status s = set_lists(b, dev_nodes, node_pre, dev_cells, cell_pre);
        if (s != HYB_OK) return s;
    }
    if (use_graph && b->stream == nullptr) {
        b->err = "graph replay needs a non-default stream";
        return HYB_ESTATE;
    }
    for (int i = 0; i < nsteps; ++i) {
        if (!use_graph) {
            const hyb_status s = batch_step(b, b->cur_p, b->cur_f);
            if (s != HYB_OK) return s;
            flip(b);
            continue;
        }
        const int gi = b->cur_p;
        if (b->graph[gi] && b->g_curf[gi] != b->cur_f) {
            cudaGraphExecDestroy(b->graph[gi]);
            b->graph[gi] = nullptr;
        }
        if (!b->graph[gi]) {
            cudaGraph_t g = nullptr;
            hyb_status s = bcheck(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                                  "begin capture");
            if (s != HYB_OK) return s;
            const hyb_status s2 = batch_step(b, b->cur_p, b->cur_f);
            cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            if (s2 != HYB_OK) {
                if (g) cudaGraphDestroy(g);
                return s2;
            }
            s = bcheck(b, e, "end capture");
            if (s != HYB_OK) return s;
            e = cudaGraphInstantiate(&b->graph[gi], g, 0);
            cudaGraphDestroy(g);
            s = bcheck(b, e, "graph instantiate");
            if (s != HYB_OK) return s;
            b->g_curf[gi] = b->cur_f;
        }
        const hyb_status s = bcheck(b, cudaGraphLaunch(b->graph[gi], b->stream), "graph launch");
        if (s != HYB_OK) return s;
        flip(b);
    }
    return HYB_OK;
}

namespace {
// Block sizes each kernel class of the batch may take (0 ends a list): the collide 32 or 16
// cells of 8 lanes per block; LB2DSMC one, fixed by its design (8 warps per cell).
const int kShapes[5][4] = {{64, 128, 256, 0}, {256, 128, 0, 0}, {32, 64, 128, 0}, {64, 128, 256, 0},
                           {256, 0, 0, 0}};
int* block_of(hyb_batch* b, int kernel) {
    switch (kernel) {
        case hyb::K_MOVE: return &b->dev.move_block;
        case hyb::K_COLLIDE: return &b->dev.collide_block;
        case hyb::K_LBM: return &b->dev.lbm_block;
        case hyb::K_D2L: return &b->dev.d2l_block;
        default: return nullptr;
    }
}
bool shape_ok(int kernel, int threads) {
    if (kernel < 0 || kernel > 4) return false;
    for (int i = 0; i < 4 && kShapes[kernel][i]; ++i)
        if (kShapes[kernel][i] == threads) return true;
    return false;
}
}  // namespace

hyb_status hyb_batch_set_block(hyb_batch* b, int32_t kernel, int32_t threads) {
    if (!b || !shape_ok(kernel, threads)) return HYB_EINVAL;
    int* p = block_of(b, kernel);
    if (p && *p != threads) {
        *p = threads;
        drop_graphs(b);
    }
    return HYB_OK;
}

int32_t hyb_batch_get_block(const hyb_batch* b, int32_t kernel) {
    if (!b || kernel < 0 || kernel > 4) return -1;
    int* p = block_of(const_cast<hyb_batch*>(b), kernel);
    return p ? *p : kShapes[kernel][0];
}

hyb_status hyb_batch_set_blocks(hyb_batch* b, int32_t move_block, int32_t lbm_block) {
    if (!b || !shape_ok(hyb::K_MOVE, move_block) || !shape_ok(hyb::K_LBM, lbm_block)) return HYB_EINVAL;
    hyb_status s = hyb_batch_set_block(b, hyb::K_MOVE, move_block);
    if (s == HYB_OK) s = hyb_batch_set_block(b, hyb::K_LBM, lbm_block);
    return s;
}

hyb_status hyb_batch_tune(hyb_batch* b, const int32_t* dev_nodes, const int64_t* node_pre,
                          const int32_t* dev_cells, const int64_t* cell_pre, int32_t* move_block,
                          int32_t* lbm_block) {
    if (!b) return HYB_EINVAL;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HYB_ECUDA;
    // the best of three replays of two hybrid steps from a captured graph
    auto time_steps = [&](float* ms) -> hyb_status {
        hyb_status s = hyb_batch_hybrid_step(b, dev_nodes, node_pre, dev_cells, cell_pre, 1, 1);  // capture
        if (s != HYB_OK) return s;
        float best = 1e30f;
        for (int k = 0; k < 3; ++k) {
            cudaEventRecord(e0, b->stream);
            s = hyb_batch_hybrid_step(b, dev_nodes, node_pre, dev_cells, cell_pre, 2, 1);
            if (s != HYB_OK) return s;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return HYB_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < best) best = t;
        }
        *ms = best;
        return HYB_OK;
    };
    // one kernel class at a time, the others at their current shapes: move, collide, LB,
    // DSMC2LB
    hyb_status s = HYB_OK;
    const int order[4] = {hyb::K_MOVE, hyb::K_COLLIDE, hyb::K_LBM, hyb::K_D2L};
    for (int ki = 0; ki < 4 && s == HYB_OK; ++ki) {
        const int k = order[ki];
        int best_t = hyb_batch_get_block(b, k);
        float best = 1e30f;
        for (int i = 0; i < 4 && kShapes[k][i] && s == HYB_OK; ++i) {
            float t = 0.f;
            s = hyb_batch_set_block(b, k, kShapes[k][i]);
            if (s == HYB_OK) s = time_steps(&t);
            if (s == HYB_OK && t < best) {
                best = t;
                best_t = kShapes[k][i];
            }
        }
        if (s == HYB_OK) s = hyb_batch_set_block(b, k, best_t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != HYB_OK) return s;
    if (move_block) *move_block = b->dev.move_block;
    if (lbm_block) *lbm_block = b->dev.lbm_block;
    return s;
}

const char* hyb_batch_last_error(const hyb_batch* b) { return b ? b->err.c_str() : "null batch"; }

void hyb_batch_destroy(hyb_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (hyb_ctx* h : b->reps) hyb_destroy(h);
    delete b;
}

}  // extern "C"
