// Host runtime of the DSMC-LBM library: parameter validation, derived constants, arena
// layout, context lifetime, launch sequencing, CUDA-graph replay of a hybrid step, kernel
// timing and error reporting. Every entry point of include/dsmclbm.h is defined here.
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <vector>
#include <utility>

#include "hyb_internal.cuh"

using namespace hyb;

namespace {

const double kPi = 3.14159265358979323846;
const double kBoltzmann = 1.380649e-23;

bool params_valid(const hyb_params* p) {
    if (!p || p->abi_version != HYB_ABI_VERSION) return false;
    if (p->ncx < 6 || p->ncy < 1 || (p->lb_ratio != 1 && p->lb_ratio != 2) || p->ppc < 1) return false;
    if (p->lattice != 39 && p->lattice != 19) return false;
    if (p->real_bytes != 4 && p->real_bytes != 8) return false;
    if (p->sample_every < 1) return false;
    if ((p->lb_collision != 0 && p->lb_collision != 1) || (p->d2l_mode != 0 && p->d2l_mode != 1))
        return false;
    if (p->kn_profile != 0 && p->kn_profile != 1) return false;
    if (p->kn_profile == 1 && !(p->kn_end > 0.0)) return false;
    if (p->ncz < 0) return false;
    if (p->accum_mode != 0) return false;  // only FP64 moment sums are built
    if (p->ncy_global < 0) return false;
    if (p->ncy_global > 0) {  // a streamwise slab of a channel of ncy_global rows
        if (p->y0 < 0 || p->ncy < 4 || (int64_t)p->y0 + p->ncy > p->ncy_global) return false;
        if (p->kn_profile == 1 && p->ncy_global < 2) return false;
    } else if (p->y0 != 0) {
        return false;
    }
    if (!(p->kn > 0.0) || !(p->crmax_init > 0.0) || !(p->capacity_factor >= 1.0)) return false;
    if (!(p->ma >= 0.0) || !(p->T_K > 0.0) || !(p->mass_kg > 0.0)) return false;
    if (std::ceil(p->capacity_factor * (double)p->ppc) > 256.0) return false;  // bin <= 256
    const double rows = p->ncy_global > 0 ? (double)p->ncy_global : (double)p->ncy;
    const double slots = (double)p->ncx * rows * (double)(p->ncz >= 2 ? p->ncz : 1) * 256.0;
    if (slots >= 2147483648.0) return false;  // origin slots fit the 31 bits of an order key
    return true;
}

// Same definitions as the derived-constant list in dsmclbm.h: Eq. tau, Eq. MFP in cell
// units, the NTC factor of Eq. collisionnumber, and the no-slip parabola of Sec. 3.1.
void derive(const hyb_params& p, hyb_derived& d) {
    std::memset(&d, 0, sizeof(d));
    d.r_lat = (p.lattice == 39) ? std::sqrt(1.5) : std::sqrt(3.0);
    d.cs_lat = 1.0 / d.r_lat;
    d.H_lat = (double)p.ncx * (double)p.lb_ratio;
    d.tau = std::sqrt(kPi / 8.0) * d.r_lat * p.kn * d.H_lat + 0.5;
    d.dt = d.cs_lat / (double)p.lb_ratio;
    d.lambda = p.kn * (double)p.ncx;
    d.coll_dt = d.dt / (std::sqrt(2.0) * d.lambda * (double)p.ppc);
    d.g_step = 8.0 * (d.tau - 0.5) * p.ma * d.cs_lat * d.cs_lat / (d.H_lat * d.H_lat);
    d.c_th_ms = std::sqrt(kBoltzmann * p.T_K / p.mass_kg);
    // 3D when ncz >= 2: cells (iz ncy + iy) ncx + ix, nodes (z ny + y) nx + x
    d.ncz = p.ncz >= 2 ? p.ncz : 1;
    d.ncells = (int64_t)p.ncx * p.ncy * d.ncz;
    d.nx = (int64_t)p.ncx * p.lb_ratio;
    // a slab's lattice has yh ghost rows below and above its own rows
    d.yh = p.ncy_global > 0 ? (p.lattice == 39 ? 3 : 1) : 0;
    d.ny = (int64_t)p.ncy * p.lb_ratio + 2 * d.yh;
    d.nz = p.ncz >= 2 ? d.ncz * p.lb_ratio : 1;
    d.nnodes = d.nx * d.ny * d.nz;
    d.bin = ((int32_t)std::ceil(p.capacity_factor * (double)p.ppc) + 31) / 32 * 32;
    d.capacity = d.ncells * (int64_t)d.bin;
    d.xcap = p.ncy_global > 0 ? (int64_t)p.ncx * d.ncz * d.bin : 0;
    d.q = p.lattice;
    d.order = (p.lattice == 39) ? 3 : 2;
}

void layout(const hyb_params& p, const hyb_derived& d, hyb_layout& L) {
    std::memset(&L, 0, sizeof(L));
    const uint64_t rb = (uint64_t)p.real_bytes;
    const uint64_t cap = (uint64_t)d.capacity, nc = (uint64_t)d.ncells, nn = (uint64_t)d.nnodes;
    const uint64_t q = (uint64_t)d.q;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = (off + bytes + 255) & ~255ull;
        return o;
    };
    for (int h = 0; h < 2; ++h) L.part[h] = take(cap * (uint64_t)kRec * rb);
    L.count[0] = take(nc * 4);
    L.count[1] = take(nc * 4);
    L.crmax = take(nc * rb);
    L.rem = take(nc * rb);
    L.nbar_sum = take(nc * 4);
    L.acc = take(nc * kMoments * 8);
    for (int h = 0; h < 2; ++h) L.f[h] = take(q * nn * rb);
    L.ctrl = take(CTRL_WORDS * 4);
    L.counters = take(HYB_NCOUNTERS * 8);
    L.map_scratch = take(nc * sizeof(GradRec));
    L.coupled = take(nc);
    // a slab's exchange buffers: a count, xcap records, xcap cell ids
    L.xbytes = d.xcap > 0 ? 256 + (uint64_t)d.xcap * ((uint64_t)kRec * rb + 4) : 0;
    for (int h = 0; h < 2; ++h) L.xsend[h] = take(L.xbytes);
    for (int h = 0; h < 2; ++h) L.xrecv[h] = take(L.xbytes);
    const bool prof = p.kn_profile == 1;
    L.coll_cell = take(prof ? nc * rb : 0);
    L.tau_node = take(prof ? nn * rb : 0);
    L.total_bytes = off;
    L.capacity = d.capacity;
    L.ncells = d.ncells;
    L.nnodes = d.nnodes;
    L.q = d.q;
    L.real_bytes = p.real_bytes;
    L.bin = d.bin;
}

// Kn along the channel (kn_profile = 1): log-linear in the streamwise coordinate y (cell
// units, period the channel's rows) from kn at y = 0 to kn_end at half the period.
double kn_at(const hyb_params& p, double y) {
    const double period = p.ncy_global > 0 ? (double)p.ncy_global : (double)p.ncy;
    const double s = 1.0 - std::fabs(2.0 * y / period - 1.0);
    return p.kn * std::exp(s * std::log(p.kn_end / p.kn));
}

hyb_status fail(Ctx& c, hyb_status s, const char* what, cudaError_t e = cudaSuccess) {
    c.err = what;
    if (e != cudaSuccess) {
        c.err += ": ";
        c.err += cudaGetErrorString(e);
    }
    return s;
}

hyb_status check(Ctx& c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HYB_OK;
    return fail(c, HYB_ECUDA, what, e);
}

void flip_particles(Ctx& c) { c.cur_p ^= 1; }
void flip_populations(Ctx& c) { c.cur_f ^= 1; }

ProfPool& pool_of(Ctx& c) { return c.pool; }

}  // namespace

namespace hyb {

void prof_begin(Ctx& c, int k) {
    if (c.prof_kernel != k) return;
    ProfPool& P = pool_of(c);
    if (c.capturing) {
        const int s = P.capture_slot;
        if (!P.ga[s]) {
            cudaEventCreate(&P.ga[s]);
            cudaEventCreate(&P.gb[s]);
        }
        cudaEventRecordWithFlags(P.ga[s], c.stream, cudaEventRecordExternal);
        return;
    }
    if (P.used == P.a.size()) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        P.a.push_back(e0);
        P.b.push_back(e1);
    }
    cudaEventRecord(P.a[P.used], c.stream);
}

void prof_end(Ctx& c, int k) {
    if (c.prof_kernel != k) return;
    ProfPool& P = pool_of(c);
    if (c.capturing) {
        cudaEventRecordWithFlags(P.gb[P.capture_slot], c.stream, cudaEventRecordExternal);
        return;
    }
    cudaEventRecord(P.b[P.used], c.stream);
    P.used += 1;
}

}  // namespace hyb

namespace {

void resolve(Ctx& c) {
    char* a = c.arena;
    const hyb_layout& L = c.L;
    State& s = c.st;
    for (int h = 0; h < 2; ++h) {
        s.part[h] = a + L.part[h];
        s.f[h] = a + L.f[h];
        s.count[h] = (uint32_t*)(a + L.count[h]);
    }
    s.coupled = (uint8_t*)(a + L.coupled);
    for (int d = 0; d < 2; ++d) {
        s.xsend[d] = a + L.xsend[d];
        s.xrecv[d] = a + L.xrecv[d];
    }
    s.crmax = a + L.crmax;
    s.rem = a + L.rem;
    s.nbar_sum = (uint32_t*)(a + L.nbar_sum);
    s.acc = (double*)(a + L.acc);
    s.ctrl = (uint32_t*)(a + L.ctrl);
    s.counters = (unsigned long long*)(a + L.counters);
    s.grad = (GradRec*)(a + L.map_scratch);
    s.coll_cell = c.p.kn_profile == 1 ? a + L.coll_cell : nullptr;
    s.tau_node = c.p.kn_profile == 1 ? a + L.tau_node : nullptr;
}

hyb_status do_dsmc_step(Ctx& c) {
    hyb_status s = check(c, launch_dsmc_step(c), "dsmc_step launch");
    if (s == HYB_OK) flip_particles(c);
    return s;
}

hyb_status do_lbm_step(Ctx& c) {
    hyb_status s = check(c, launch_lbm_step(c), "lbm_step launch");
    if (s == HYB_OK) flip_populations(c);
    return s;
}

// n DSMC steps: the move of the first, then n - 1 fused passes (the collide of one step and
// the move of the next), then the collide of the last. The particle parity flips once per step.
// Whether multi-step calls fuse the DSMC passes (HYB_FUSE_AUTO: when the fused grid fills the
// GPU). Either way the results are the same bit for bit.
bool fuse_steps(Ctx& c) {
    if (c.fuse_mode == HYB_FUSE_ALWAYS) return true;
    if (c.fuse_mode == HYB_FUSE_NEVER) return false;
    if (c.fuse_pays < 0) c.fuse_pays = dsmc_fused_fills_gpu(c) ? 1 : 0;
    return c.fuse_pays == 1;
}

hyb_status one_hybrid_step(Ctx& c, const int32_t* nodes, int32_t nn, const int32_t* cells, int32_t ncl);

hyb_status dsmc_steps(Ctx& c, int n) {
    if (n <= 0) return HYB_OK;
    if (n > 1 && !fuse_steps(c)) {
        hyb_status s = HYB_OK;
        for (int k = 0; k < n && s == HYB_OK; ++k) s = do_dsmc_step(c);
        return s;
    }
    int p = c.cur_p;
    hyb_status s = check(c, launch_dsmc_move(c, p), "dsmc move launch");
    for (int k = 1; k < n && s == HYB_OK; ++k) {
        s = check(c, launch_dsmc_fused(c, p), "dsmc fused launch");
        p ^= 1;
    }
    if (s == HYB_OK) s = check(c, launch_dsmc_collide(c, p), "dsmc collide launch");
    if (s == HYB_OK) c.cur_p = p ^ 1;
    return s;
}

// Work a caller adds around each step of a multi-step call: before step k >= 1 (ahead of its
// first kernel) and after step k's LB2DSMC, on the context's stream.
struct StepHooks {
    std::function<hyb_status(int)> before, after;
};

// n hybrid steps in the order of one_hybrid_step, with the DSMC passes fused across steps:
// move; then per step the fused pass (the last step: the collide), DSMC2LB, the LB step and
// LB2DSMC, which within the fused run regenerates the coupling cells and moves their new
// particles on at once. The coupling cells are marked for the fused passes for the call's
// duration. The results equal n calls of one_hybrid_step bit for bit.
hyb_status fused_hybrid_steps(Ctx& c, const int32_t* nodes, int32_t nn, const int32_t* cells,
                              int32_t ncl, int n, const StepHooks* hk = nullptr) {
    if (n <= 0) return HYB_OK;
    if (n > 1 && !fuse_steps(c)) {
        hyb_status s = HYB_OK;
        for (int k = 0; k < n && s == HYB_OK; ++k) {
            if (hk && k > 0) s = hk->before(k);
            if (s == HYB_OK) s = one_hybrid_step(c, nodes, nn, cells, ncl);
            if (s == HYB_OK && hk) s = hk->after(k);
        }
        return s;
    }
    int p = c.cur_p;
    hyb_status s = HYB_OK;
    const bool mark = ncl > 0 && n > 1;
    if (mark) s = check(c, launch_mark_cells(c, cells, ncl, 1), "mark coupling cells");
    if (s == HYB_OK) s = check(c, launch_dsmc_move(c, p), "dsmc move launch");
    for (int k = 0; k < n && s == HYB_OK; ++k) {
        const bool last = k == n - 1;
        if (hk && k > 0) s = hk->before(k);
        if (s != HYB_OK) break;
        s = last ? check(c, launch_dsmc_collide(c, p), "dsmc collide launch")
                 : check(c, launch_dsmc_fused(c, p), "dsmc fused launch");
        if (s == HYB_OK && nn > 0) s = check(c, launch_map_d2l(c, nodes, nn), "map_dsmc_to_lbm launch");
        if (s == HYB_OK) s = do_lbm_step(c);
        if (s != HYB_OK) break;
        if (last) {
            c.cur_p = p ^ 1;
            if (ncl > 0) s = check(c, launch_map_l2d(c, cells, ncl), "map_lbm_to_dsmc launch");
        } else {
            if (ncl > 0) s = check(c, launch_map_l2d_move(c, cells, ncl, p), "map_lbm_to_dsmc launch");
            p ^= 1;
        }
        if (s == HYB_OK && hk) s = hk->after(k);
    }
    if (s == HYB_OK && mark) s = check(c, launch_mark_cells(c, cells, ncl, 0), "clear coupling cells");
    return s;
}

hyb_status one_hybrid_step(Ctx& c, const int32_t* nodes, int32_t nn, const int32_t* cells,
                           int32_t ncl) {
    hyb_status s = do_dsmc_step(c);
    if (s != HYB_OK) return s;
    if (nn > 0) {
        s = check(c, launch_map_d2l(c, nodes, nn), "map_dsmc_to_lbm launch");
        if (s != HYB_OK) return s;
    }
    s = do_lbm_step(c);
    if (s != HYB_OK) return s;
    if (ncl > 0) s = check(c, launch_map_l2d(c, cells, ncl), "map_lbm_to_dsmc launch");
    return s;
}

// The per-cell NTC factor (Eq. collisionnumber at the cell's Kn) and per-node relaxation
// time (Eq. tau at the node's Kn), formed on the host in FP64 and copied to the arena.
hyb_status fill_kn_profile(Ctx& c) {
    const int64_t nc = c.d.ncells, nn = c.d.nnodes;
    std::vector<double> cell(nc), node(nn);
    for (int64_t k = 0; k < nc; ++k) {
        // the channel's row of the cell (a slab's rows start at y0)
        const double kn = kn_at(c.p, (double)(c.p.y0 + (k / c.p.ncx) % c.p.ncy) + 0.5);
        cell[k] = c.d.dt / (std::sqrt(2.0) * (kn * (double)c.p.ncx) * (double)c.p.ppc);
    }
    for (int64_t k = 0; k < nn; ++k) {
        // the channel's LB row of the node (a slab's ghost rows hold its neighbours' rows)
        int64_t row = (int64_t)c.p.y0 * c.p.lb_ratio + (k / c.d.nx) % c.d.ny - c.d.yh;
        const int64_t nrows = (int64_t)(c.p.ncy_global > 0 ? c.p.ncy_global : c.p.ncy) * c.p.lb_ratio;
        row = ((row % nrows) + nrows) % nrows;
        const double kn = kn_at(c.p, ((double)row + 0.5) / (double)c.p.lb_ratio);
        node[k] = std::sqrt(kPi / 8.0) * c.d.r_lat * kn * c.d.H_lat + 0.5;
    }
    auto put = [&](const std::vector<double>& v, void* dst) {
        if (c.p.real_bytes == 8) return cudaMemcpy(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice);
        std::vector<float> w(v.begin(), v.end());
        return cudaMemcpy(dst, w.data(), w.size() * 4, cudaMemcpyHostToDevice);
    };
    hyb_status s = check(c, put(cell, c.st.coll_cell), "kn profile copy");
    if (s == HYB_OK) s = check(c, put(node, c.st.tau_node), "kn profile copy");
    return s;
}

void drop_graphs(Ctx& c) {
    for (int i = 0; i < 2; ++i) {
        if (c.graph[i]) {
            cudaGraphExecDestroy(c.graph[i]);
            c.graph[i] = nullptr;
        }
        if (c.mgraph[i]) {
            cudaGraphExecDestroy(c.mgraph[i]);
            c.mgraph[i] = nullptr;
        }
        c.mkey[i][0] = c.mkey[i][1] = c.mkey[i][2] = -1;
        if (c.hgraph[i]) {
            cudaGraphExecDestroy(c.hgraph[i]);
            c.hgraph[i] = nullptr;
        }
        c.hkey[i] = Ctx::HostKey{};
    }
}

// A multi-step fused hybrid call replayed from a graph captured on first use (per step
// count and starting parities; the lists and profiling state are checked by the caller).
hyb_status fused_graph_run(Ctx& c, const int32_t* nodes, int32_t nn, const int32_t* cells, int32_t ncl,
                           int n) {
    int slot = -1;
    for (int i = 0; i < 2; ++i)
        if (c.mgraph[i] && c.mkey[i][0] == n && c.mkey[i][1] == c.cur_p && c.mkey[i][2] == c.cur_f)
            slot = i;
    const int cp = c.cur_p, cf = c.cur_f;
    if (slot < 0) {
        slot = c.mnext;
        c.mnext ^= 1;
        if (c.mgraph[slot]) {
            cudaGraphExecDestroy(c.mgraph[slot]);
            c.mgraph[slot] = nullptr;
        }
        cudaGraph_t g = nullptr;
        hyb_status s = check(c, cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal),
                             "begin capture");
        if (s != HYB_OK) return s;
        c.capturing = true;
        hyb_status s2 = fused_hybrid_steps(c, nodes, nn, cells, ncl, n);
        c.capturing = false;
        cudaError_t e = cudaStreamEndCapture(c.stream, &g);
        c.cur_p = cp;
        c.cur_f = cf;
        if (s2 != HYB_OK) {
            if (g) cudaGraphDestroy(g);
            return s2;
        }
        s = check(c, e, "end capture");
        if (s != HYB_OK) return s;
        e = cudaGraphInstantiate(&c.mgraph[slot], g, 0);
        cudaGraphDestroy(g);
        s = check(c, e, "graph instantiate");
        if (s != HYB_OK) return s;
        c.mkey[slot][0] = n;
        c.mkey[slot][1] = cp;
        c.mkey[slot][2] = cf;
    }
    hyb_status s = check(c, cudaGraphLaunch(c.mgraph[slot], c.stream), "graph launch");
    if (s != HYB_OK) return s;
    // each step flips both parities once
    c.cur_p = cp ^ (n & 1);
    c.cur_f = cf ^ (n & 1);
    return HYB_OK;
}

}  // namespace

extern "C" {

const char* hyb_status_string(hyb_status s) {
    switch (s) {
        case HYB_OK: return "ok";
        case HYB_EINVAL: return "invalid argument";
        case HYB_ENOMEM: return "arena too small";
        case HYB_ECUDA: return "CUDA error";
        case HYB_ECAPACITY: return "capacity exceeded";
        case HYB_ETIMEOUT: return "capped device loop reached its limit";
        case HYB_ESAMPLING: return "acceptance-rejection attempt cap reached";
        case HYB_ESTATE: return "call out of order";
    }
    return "unknown status";
}

hyb_status hyb_derive(const hyb_params* p, hyb_derived* out) {
    if (!params_valid(p) || !out) return HYB_EINVAL;
    derive(*p, *out);
    return HYB_OK;
}

hyb_status hyb_layout_compute(const hyb_params* p, hyb_layout* out) {
    if (!params_valid(p) || !out) return HYB_EINVAL;
    hyb_derived d;
    derive(*p, d);
    layout(*p, d, *out);
    return HYB_OK;
}

hyb_status hyb_lattice(int32_t q, int32_t* e, double* w, double* r) {
    if ((q != 39 && q != 19) || !e || !w || !r) return HYB_EINVAL;
    if (q == 39) {
        for (int a = 0; a < 39; ++a) {
            for (int i = 0; i < 3; ++i) e[3 * a + i] = LatTab<D3Q39>::e(a, i);
            w[a] = LatTab<D3Q39>::w(a);
        }
        *r = lat_r<D3Q39>();
    } else {
        for (int a = 0; a < 19; ++a) {
            for (int i = 0; i < 3; ++i) e[3 * a + i] = LatTab<D3Q19>::e(a, i);
            w[a] = LatTab<D3Q19>::w(a);
        }
        *r = lat_r<D3Q19>();
    }
    return HYB_OK;
}

hyb_status dsmc_init(const hyb_params* p, void* arena, uint64_t arena_bytes, void* stream,
                     hyb_ctx** out) {
    if (!out || !params_valid(p) || !arena || ((uintptr_t)arena & 255u)) return HYB_EINVAL;
    *out = nullptr;
    hyb_ctx* h = new (std::nothrow) hyb_ctx();
    if (!h) return HYB_ENOMEM;
    Ctx& c = h->c;
    c.p = *p;
    derive(c.p, c.d);
    layout(c.p, c.d, c.L);
    if (arena_bytes < c.L.total_bytes) {
        delete h;
        return HYB_ENOMEM;
    }
    c.arena = (char*)arena;
    c.stream = (cudaStream_t)stream;
    resolve(c);
    cudaGetDevice(&c.device);
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
    // pinned host words for status reads, followed by the timing pool
    void* hp = nullptr;
    if (cudaMallocHost(&hp, 256) != cudaSuccess) {
        delete h;
        return HYB_ECUDA;
    }
    c.h_pinned = (uint32_t*)hp;
    hyb_status s = check(c, launch_init(c), "dsmc_init launch");
    if (s == HYB_OK && c.p.kn_profile == 1) s = fill_kn_profile(c);
    if (s != HYB_OK) {
        cudaFreeHost(hp);
        delete h;
        return s;
    }
    *out = h;
    return HYB_OK;
}

hyb_status dsmc_step(hyb_ctx* h, int32_t nsteps) {
    if (!h || nsteps < 0) return HYB_EINVAL;
    if (h->c.p.ncy_global > 0 || h->c.split_pending)
        return fail(h->c, HYB_EINVAL, "dsmc_step: a slab steps with dsmc_move, dsmc_merge and dsmc_collide");
    return dsmc_steps(h->c, nsteps);
}

hyb_status dsmc_move(hyb_ctx* h) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    if (c.split_pending) return fail(c, HYB_ESTATE, "dsmc_move: the previous move has no collide yet");
    hyb_status s = check(c, launch_dsmc_move(c, c.cur_p), "dsmc_move launch");
    if (s == HYB_OK) c.split_pending = true;
    return s;
}

hyb_status dsmc_merge(hyb_ctx* h) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    if (!c.split_pending) return fail(c, HYB_ESTATE, "dsmc_merge: no move to merge into");
    return check(c, launch_dsmc_merge(c, c.cur_p), "dsmc_merge launch");
}

hyb_status dsmc_collide(hyb_ctx* h) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    if (!c.split_pending) return fail(c, HYB_ESTATE, "dsmc_collide: no move to collide");
    hyb_status s = check(c, launch_dsmc_collide(c, c.cur_p), "dsmc_collide launch");
    if (s == HYB_OK) {
        c.split_pending = false;
        flip_particles(c);
    }
    return s;
}

hyb_status lbm_halo_size(const hyb_ctx* h, int64_t* values) {
    if (!h || !values || h->c.d.yh == 0) return HYB_EINVAL;
    *values = lbm_halo_values(h->c);
    return HYB_OK;
}

hyb_status lbm_halo_pack(hyb_ctx* h, int32_t side, void* dev_buf) {
    if (!h || !dev_buf || (side != 0 && side != 1) || h->c.d.yh == 0) return HYB_EINVAL;
    return check(h->c, launch_lbm_halo(h->c, side, dev_buf, 0), "lbm_halo_pack launch");
}

hyb_status lbm_halo_unpack(hyb_ctx* h, int32_t side, const void* dev_buf) {
    if (!h || !dev_buf || (side != 0 && side != 1) || h->c.d.yh == 0) return HYB_EINVAL;
    return check(h->c, launch_lbm_halo(h->c, side, (void*)dev_buf, 1), "lbm_halo_unpack launch");
}

hyb_status lbm_step(hyb_ctx* h, int32_t nsteps) {
    if (!h || nsteps < 0) return HYB_EINVAL;
    for (int i = 0; i < nsteps; ++i) {
        hyb_status s = do_lbm_step(h->c);
        if (s != HYB_OK) return s;
    }
    return HYB_OK;
}

hyb_status sample_moments(hyb_ctx* h, double* out, int32_t reset) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    const size_t bytes = (size_t)c.d.ncells * kMoments * sizeof(double);
    if (out) {
        hyb_status s = check(c, cudaMemcpyAsync(out, c.st.acc, bytes, cudaMemcpyDeviceToDevice,
                                                c.stream), "sample_moments copy");
        if (s != HYB_OK) return s;
    }
    if (reset) {
        hyb_status s = check(c, cudaMemsetAsync(c.st.acc, 0, bytes, c.stream), "reset sums");
        if (s != HYB_OK) return s;
        s = check(c, cudaMemsetAsync(c.st.ctrl + CTRL_NSAMPLES, 0, 4, c.stream), "reset count");
        if (s != HYB_OK) return s;
    }
    return HYB_OK;
}

hyb_status map_dsmc_to_lbm(hyb_ctx* h, const int32_t* dev_nodes, int32_t n) {
    if (!h || n < 0 || (n > 0 && !dev_nodes) || n > h->c.d.nnodes) return HYB_EINVAL;
    if (n == 0) return HYB_OK;
    return check(h->c, launch_map_d2l(h->c, dev_nodes, n), "map_dsmc_to_lbm launch");
}

hyb_status map_lbm_to_dsmc(hyb_ctx* h, const int32_t* dev_cells, int32_t n) {
    if (!h || n < 0 || (n > 0 && !dev_cells) || n > h->c.d.ncells) return HYB_EINVAL;
    if (n == 0) return HYB_OK;
    return check(h->c, launch_map_l2d(h->c, dev_cells, n), "map_lbm_to_dsmc launch");
}

hyb_status lbm_step_nodes(hyb_ctx* h, const void* f_src, void* f_dst, const void* g_node,
                          const void* tau_node) {
    if (!h || !f_src || !f_dst || f_src == f_dst || !g_node || !tau_node) return HYB_EINVAL;
    return check(h->c, launch_lbm_step_nodes(h->c, f_src, f_dst, g_node, tau_node),
                 "lbm_step_nodes launch");
}

hyb_status lbm_interface_loss(hyb_ctx* h, const void* f, const int32_t* dev_nodes, int32_t n,
                              const void* dev_targets, double* dev_loss, void* lam) {
    if (!h || !f || n < 0 || (n > 0 && (!dev_nodes || !dev_targets || !dev_loss || !lam)))
        return HYB_EINVAL;
    if (n == 0) return HYB_OK;
    return check(h->c, launch_interface_loss(h->c, f, dev_nodes, n, dev_targets, dev_loss, lam),
                 "lbm_interface_loss launch");
}

hyb_status lbm_adjoint_step(hyb_ctx* h, const void* f, const void* lam_next, void* lam,
                            const void* g_node, const void* tau_node, void* grad_g,
                            void* grad_tau, void* wall) {
    if (!h || !f || !lam_next || !lam || lam == lam_next || !g_node || !tau_node || !grad_g ||
        !grad_tau || !wall || h->c.p.lb_collision != 0)
        return HYB_EINVAL;
    return check(h->c, launch_lbm_adjoint_step(h->c, f, lam_next, lam, g_node, tau_node, grad_g,
                                               grad_tau, wall),
                 "lbm_adjoint_step launch");
}

hyb_status lbm_steps_nodes(hyb_ctx* h, void* f_a, void* f_b, const void* g_node, const void* tau_node,
                           int32_t nsteps, int32_t ckpt_every, void* ckpt) {
    if (!h || !f_a || !f_b || f_a == f_b || !g_node || !tau_node || nsteps < 0 || ckpt_every < 1)
        return HYB_EINVAL;
    const int32_t nck = nsteps > 0 ? (nsteps - 1) / ckpt_every : 0;
    if (nck > 0 && !ckpt) return HYB_EINVAL;
    Ctx& c = h->c;
    const size_t bytes = (size_t)c.d.q * (size_t)c.d.nnodes * (size_t)c.p.real_bytes;
    void* src = f_a;
    void* dst = f_b;
    for (int32_t t = 0; t < nsteps; ++t) {
        hyb_status s = check(c, launch_lbm_step_nodes(c, src, dst, g_node, tau_node), "lbm_steps_nodes launch");
        if (s != HYB_OK) return s;
        std::swap(src, dst);
        if ((t + 1) % ckpt_every == 0 && t + 1 < nsteps) {
            char* out = (char*)ckpt + (size_t)((t + 1) / ckpt_every - 1) * bytes;
            s = check(c, cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, c.stream), "checkpoint copy");
            if (s != HYB_OK) return s;
        }
    }
    return HYB_OK;
}

hyb_status lbm_adjoint_segment(hyb_ctx* h, const void* state0, void* states, int32_t n, void* lam_a,
                               void* lam_b, const void* g_node, const void* tau_node, void* grad_g,
                               void* grad_tau, void* wall) {
    if (!h || !state0 || n < 1 || (n > 1 && !states) || !lam_a || !lam_b || lam_a == lam_b || !g_node ||
        !tau_node || !grad_g || !grad_tau || !wall || h->c.p.lb_collision != 0)
        return HYB_EINVAL;
    Ctx& c = h->c;
    const size_t bytes = (size_t)c.d.q * (size_t)c.d.nnodes * (size_t)c.p.real_bytes;
    // f_t0 + k for k = 0 .. n - 1: the given state, then the recomputed ones
    auto state = [&](int32_t k) -> const void* {
        return k == 0 ? state0 : (const void*)((const char*)states + (size_t)(k - 1) * bytes);
    };
    for (int32_t k = 1; k < n; ++k) {
        hyb_status s = check(c, launch_lbm_step_nodes(c, state(k - 1), (void*)state(k), g_node, tau_node),
                             "lbm_adjoint_segment recompute");
        if (s != HYB_OK) return s;
    }
    void* next = lam_a;
    void* cur = lam_b;
    for (int32_t k = n - 1; k >= 0; --k) {
        hyb_status s = check(c, launch_lbm_adjoint_step(c, state(k), next, cur, g_node, tau_node, grad_g,
                                                        grad_tau, wall),
                             "lbm_adjoint_segment step");
        if (s != HYB_OK) return s;
        std::swap(next, cur);
    }
    return HYB_OK;
}

hyb_status map_dsmc_to_lbm_adjoint(hyb_ctx* h, const int32_t* dev_nodes, int32_t n, void* lam,
                                   double* grad_acc) {
    if (!h || n < 0 || (n > 0 && (!dev_nodes || !lam || !grad_acc)) || n > h->c.d.nnodes ||
        h->c.p.d2l_mode != 0)
        return HYB_EINVAL;
    if (n == 0) return HYB_OK;
    return check(h->c, launch_map_d2l_adjoint(h->c, dev_nodes, n, lam, grad_acc),
                 "map_dsmc_to_lbm_adjoint launch");
}

hyb_status map_lbm_to_dsmc_noalloc(hyb_ctx* h, const int32_t* dev_cells, int32_t n) {
    if (!h || n < 0 || (n > 0 && !dev_cells) || n > h->c.d.ncells) return HYB_EINVAL;
    Ctx& c = h->c;
    if (n > HYB_NOALLOC_MAX_CELLS)
        return fail(c, HYB_EINVAL,
                    "map_lbm_to_dsmc_noalloc: more coupling cells than its fixed scratch holds "
                    "(HYB_NOALLOC_MAX_CELLS)");
    if (n == 0) return HYB_OK;
    const cudaError_t e = launch_map_l2d_noalloc(c, dev_cells, n);
    if (e == cudaErrorInvalidDevice)
        return fail(c, HYB_EINVAL,
                    "map_lbm_to_dsmc_noalloc: the context's device must be the current device", e);
    return check(c, e, "map_lbm_to_dsmc_noalloc launch");
}

hyb_status hyb_hybrid_step(hyb_ctx* h, const int32_t* dev_nodes, int32_t n_nodes,
                           const int32_t* dev_cells, int32_t n_cells, int32_t nsteps,
                           int32_t use_graph) {
    if (!h || nsteps < 0 || n_nodes < 0 || n_cells < 0) return HYB_EINVAL;
    Ctx& c = h->c;
    if (c.p.ncy_global > 0 || c.split_pending)
        return fail(c, HYB_EINVAL, "hyb_hybrid_step: a slab steps with the split calls");
    if ((n_nodes > 0 && !dev_nodes) || (n_cells > 0 && !dev_cells) || n_nodes > c.d.nnodes ||
        n_cells > c.d.ncells)
        return HYB_EINVAL;
    if (!use_graph) return fused_hybrid_steps(c, dev_nodes, n_nodes, dev_cells, n_cells, nsteps);
    if (c.stream == nullptr) return fail(c, HYB_ESTATE, "graph replay needs a non-default stream");
    if (c.g_nodes != dev_nodes || c.g_cells != dev_cells || c.g_nn != n_nodes ||
        c.g_nc != n_cells || c.g_prof != c.prof_kernel) {
        drop_graphs(c);
        c.g_nodes = dev_nodes;
        c.g_cells = dev_cells;
        c.g_nn = n_nodes;
        c.g_nc = n_cells;
        c.g_prof = c.prof_kernel;
    }
    // several steps with no kernel timing: one graph of the fused run
    if (nsteps > 1 && c.prof_kernel < 0)
        return fused_graph_run(c, dev_nodes, n_nodes, dev_cells, n_cells, nsteps);
    ProfPool& P = pool_of(c);
    for (int i = 0; i < nsteps; ++i) {
        // The graph variant is fixed by the particle parity; the population parity flips in
        // step with it inside a hybrid step, so it is recorded at capture and checked.
        const int gi = c.cur_p;
        if (!c.graph[gi]) {
            const int save_p = c.cur_p, save_f = c.cur_f;
            cudaGraph_t g = nullptr;
            hyb_status s = check(c, cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal),
                                 "begin capture");
            if (s != HYB_OK) return s;
            c.capturing = true;
            P.capture_slot = gi * 2 + c.cur_f;
            hyb_status s2 = one_hybrid_step(c, dev_nodes, n_nodes, dev_cells, n_cells);
            c.capturing = false;
            cudaError_t e = cudaStreamEndCapture(c.stream, &g);
            c.cur_p = save_p;
            c.cur_f = save_f;
            if (s2 != HYB_OK) {
                if (g) cudaGraphDestroy(g);
                return s2;
            }
            s = check(c, e, "end capture");
            if (s != HYB_OK) return s;
            e = cudaGraphInstantiate(&c.graph[gi], g, 0);
            cudaGraphDestroy(g);
            s = check(c, e, "graph instantiate");
            if (s != HYB_OK) return s;
            c.g_prof = c.prof_kernel;
            c.g_curf[gi] = c.cur_f;
        }
        if (c.g_curf[gi] != c.cur_f) {
            // population parity differs from the captured one: recapture this variant
            cudaGraphExecDestroy(c.graph[gi]);
            c.graph[gi] = nullptr;
            --i;
            continue;
        }
        hyb_status s = check(c, cudaGraphLaunch(c.graph[gi], c.stream), "graph launch");
        if (s != HYB_OK) return s;
        if (c.prof_kernel >= 0) P.gpending[gi * 2 + c.cur_f] = true;
        flip_particles(c);
        flip_populations(c);
    }
    return HYB_OK;
}

hyb_status hyb_set_collide_block(hyb_ctx* h, int32_t warps) {
    if (!h || (warps != 4 && warps != 8)) return HYB_EINVAL;
    if (h->c.collide_warps != warps) {
        h->c.collide_warps = warps;
        h->c.fuse_pays = -1;  // formed again for this shape
        drop_graphs(h->c);
    }
    return HYB_OK;
}

int32_t hyb_get_collide_block(const hyb_ctx* h) { return h ? h->c.collide_warps : -1; }

hyb_status hyb_tune_collide(hyb_ctx* h, const int32_t* dev_nodes, int32_t n_nodes, const int32_t* dev_cells,
                            int32_t n_cells, int32_t* warps, int32_t* fuse) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HYB_ECUDA;
    // (block shape, fusion) pairs, each timed on captured eight-step calls: the capture call
    // and one replay untimed, then the best of four replays (short calls on small channels
    // vary by tens of percent from call to call)
    constexpr int kSteps = 8, kReplays = 4;
    const int shapes[4] = {8, 4, 8, 4};
    const int modes[4] = {HYB_FUSE_ALWAYS, HYB_FUSE_ALWAYS, HYB_FUSE_NEVER, HYB_FUSE_NEVER};
    float best = 1e30f;
    int best_i = 0;
    hyb_status s = HYB_OK;
    for (int i = 0; i < 4 && s == HYB_OK; ++i) {
        s = hyb_set_collide_block(h, shapes[i]);
        if (s == HYB_OK) s = hyb_set_fuse(h, modes[i]);
        for (int k = 0; k < 2 && s == HYB_OK; ++k)
            s = hyb_hybrid_step(h, dev_nodes, n_nodes, dev_cells, n_cells, kSteps, 1);
        float t_best = 1e30f;
        for (int k = 0; k < kReplays && s == HYB_OK; ++k) {
            cudaEventRecord(e0, c.stream);
            s = hyb_hybrid_step(h, dev_nodes, n_nodes, dev_cells, n_cells, kSteps, 1);
            cudaEventRecord(e1, c.stream);
            if (s == HYB_OK && cudaEventSynchronize(e1) != cudaSuccess) s = HYB_ECUDA;
            float t = 0.f;
            if (s == HYB_OK) cudaEventElapsedTime(&t, e0, e1);
            if (t < t_best) t_best = t;
        }
        if (s == HYB_OK && t_best < best) {
            best = t_best;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != HYB_OK) return s;
    s = hyb_set_collide_block(h, shapes[best_i]);
    if (s == HYB_OK) s = hyb_set_fuse(h, modes[best_i]);
    if (warps) *warps = shapes[best_i];
    if (fuse) *fuse = modes[best_i];
    return s;
}

hyb_status hyb_set_fuse(hyb_ctx* h, int32_t mode) {
    if (!h || mode < HYB_FUSE_AUTO || mode > HYB_FUSE_NEVER) return HYB_EINVAL;
    if (h->c.fuse_mode != mode) {
        h->c.fuse_mode = mode;
        drop_graphs(h->c);  // graphs hold the passes of the mode they were captured in
    }
    return HYB_OK;
}

hyb_status hyb_current(const hyb_ctx* h, int32_t* particle_half, int32_t* lb_half) {
    if (!h) return HYB_EINVAL;
    if (particle_half) *particle_half = h->c.cur_p;
    if (lb_half) *lb_half = h->c.cur_f;
    return HYB_OK;
}

hyb_status hyb_sync_status(hyb_ctx* h, uint32_t* bits) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    hyb_status s = check(c, cudaStreamSynchronize(c.stream), "synchronize");
    if (s != HYB_OK) return s;
    s = check(c, cudaMemcpy(c.h_pinned, c.st.ctrl, 4, cudaMemcpyDeviceToHost), "read status");
    if (s != HYB_OK) return s;
    const uint32_t b = c.h_pinned[0];
    if (bits) *bits = b;
    if (b & (HYB_ST_CAPACITY | HYB_ST_CELL_OVERFLOW)) return HYB_ECAPACITY;
    if (b & HYB_ST_SAMPLING_CAP) return HYB_ESAMPLING;
    if (b & (HYB_ST_BOUNCE_CAP | HYB_ST_SCATTER_CAP)) return HYB_ETIMEOUT;
    if (b & HYB_ST_BAD_INPUT) return HYB_EINVAL;
    return HYB_OK;
}

hyb_status hyb_read_counters(hyb_ctx* h, uint64_t* out) {
    if (!h || !out) return HYB_EINVAL;
    Ctx& c = h->c;
    hyb_status s = check(c, cudaStreamSynchronize(c.stream), "synchronize");
    if (s != HYB_OK) return s;
    return check(c, cudaMemcpy(out, c.st.counters, HYB_NCOUNTERS * 8, cudaMemcpyDeviceToHost),
                 "read counters");
}

hyb_status hyb_profile(hyb_ctx* h, int32_t kernel) {
    if (!h || kernel < -1 || kernel >= K_COUNT) return HYB_EINVAL;
    h->c.prof_kernel = kernel;
    return HYB_OK;
}

hyb_status hyb_profile_harvest(hyb_ctx* h) {
    if (!h) return HYB_EINVAL;
    Ctx& c = h->c;
    hyb_status s = check(c, cudaStreamSynchronize(c.stream), "synchronize");
    if (s != HYB_OK) return s;
    ProfPool& P = pool_of(c);
    for (size_t i = 0; i < P.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P.a[i], P.b[i]) == cudaSuccess) {
            c.prof_ms += ms;
            c.prof_launches += 1;
        }
    }
    P.used = 0;
    for (int g = 0; g < 4; ++g)
        if (P.gpending[g] && P.ga[g]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, P.ga[g], P.gb[g]) == cudaSuccess) {
                c.prof_ms += ms;
                c.prof_launches += 1;
            }
            P.gpending[g] = false;
        }
    return HYB_OK;
}

hyb_status hyb_profile_read(const hyb_ctx* h, double* total_ms, int64_t* launches) {
    if (!h) return HYB_EINVAL;
    if (total_ms) *total_ms = h->c.prof_ms;
    if (launches) *launches = h->c.prof_launches;
    return HYB_OK;
}

hyb_status hyb_debug_philox(const uint32_t* dev_ctr, uint64_t seed, uint32_t* dev_out, int64_t n,
                            void* stream) {
    if (!dev_ctr || !dev_out || n < 0) return HYB_EINVAL;
    if (n == 0) return HYB_OK;
    return launch_debug_philox(dev_ctr, seed, dev_out, n, (cudaStream_t)stream) == cudaSuccess
               ? HYB_OK
               : HYB_ECUDA;
}

const char* hyb_last_error(const hyb_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

// The device address of page-locked host memory (cudaMallocHost, cudaHostRegister), false for
// pageable memory.
static bool device_view(const void* p, void** dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
    *dev = a.devicePointer;
    return true;
}

hyb_status hyb_hybrid_step_host(hyb_ctx* h, const int32_t* host_nodes, int32_t n_nodes,
                                const int32_t* host_cells, int32_t n_cells, double* host_acc,
                                uint32_t* host_status) {
    return hyb_hybrid_steps_host(h, 1, host_nodes, n_nodes, host_cells, n_cells, host_acc, host_status);
}

hyb_status hyb_hybrid_steps_host(hyb_ctx* h, int32_t nsteps, const int32_t* host_nodes, int32_t n_nodes,
                                 const int32_t* host_cells, int32_t n_cells, double* host_acc,
                                 uint32_t* host_status) {
    if (!h || nsteps < 1 || n_nodes < 0 || n_cells < 0 || !host_status) return HYB_EINVAL;
    Ctx& c = h->c;
    if ((n_nodes > 0 && !host_nodes) || (n_cells > 0 && (!host_cells || !host_acc)) ||
        n_nodes > c.d.nnodes || n_cells > c.d.ncells)
        return HYB_EINVAL;
    if (c.p.ncy_global > 0 || c.split_pending)
        return fail(c, HYB_EINVAL, "hyb_hybrid_steps_host: a slab steps with the split calls");
    if (c.stream == nullptr) return fail(c, HYB_ESTATE, "host steps need a non-default stream");
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_c = up(4 * (size_t)n_nodes), off_a = off_c + up(4 * (size_t)n_cells);
    const size_t need = off_a + up(8 * (size_t)kMoments * n_cells) + 256;
    if (need > c.io_bytes) {
        hyb_status s = check(c, cudaStreamSynchronize(c.stream), "synchronize");
        if (s != HYB_OK) return s;
        if (c.io_dev) cudaFree(c.io_dev);
        c.io_dev = nullptr;
        c.io_bytes = 0;
        s = check(c, cudaMalloc((void**)&c.io_dev, need), "host-step staging");
        if (s != HYB_OK) return s;
        c.io_bytes = need;
    }
    for (int i = 0; i < 4; ++i)
        if (!c.io_ev[i]) {
            hyb_status s = check(c, cudaEventCreateWithFlags(&c.io_ev[i], cudaEventDisableTiming),
                                 "event create");
            if (s != HYB_OK) return s;
        }
    if (c.io_issued - c.io_done >= 4) {
        hyb_status s = hyb_host_wait(h, 3);
        if (s != HYB_OK) return s;
    }
    int32_t* dn = (int32_t*)c.io_dev;
    int32_t* dc = (int32_t*)(c.io_dev + off_c);
    double* da = (double*)(c.io_dev + off_a);
    // Page-locked host buffers are addressable from the device: a kernel reads the lists from
    // them and another writes the sums and the status word into them, so a step's transfers
    // are two kernel launches (and the call one CUDA graph). Pageable buffers take copies.
    void *vn = nullptr, *vc = nullptr, *va = nullptr, *vs = nullptr;
    const bool mapped = (n_nodes == 0 || device_view(host_nodes, &vn)) &&
                        (n_cells == 0 || (device_view(host_cells, &vc) && device_view(host_acc, &va))) &&
                        device_view(host_status, &vs);
    const int32_t* mn = (const int32_t*)vn;
    const int32_t* mc = (const int32_t*)vc;
    double* ma = (double*)va;
    uint32_t* ms = (uint32_t*)vs;
    // every step copies the lists in before its first kernel and its strip sums and status out
    auto copy_in = [&](int) -> hyb_status {
        if (mapped) return check(c, launch_lists_in(c, mn, n_nodes, mc, n_cells, dn, dc), "lists-in launch");
        hyb_status s = HYB_OK;
        if (n_nodes > 0)
            s = check(c, cudaMemcpyAsync(dn, host_nodes, 4 * (size_t)n_nodes, cudaMemcpyHostToDevice, c.stream),
                      "copy nodes in");
        if (s == HYB_OK && n_cells > 0)
            s = check(c, cudaMemcpyAsync(dc, host_cells, 4 * (size_t)n_cells, cudaMemcpyHostToDevice, c.stream),
                      "copy cells in");
        return s;
    };
    auto copy_out = [&](int k) -> hyb_status {
        if (mapped)
            return check(c, launch_results_out(c, dc, n_cells, ma ? ma + (size_t)k * kMoments * n_cells : nullptr,
                                               ms + k),
                         "results-out launch");
        hyb_status s = HYB_OK;
        if (n_cells > 0) s = check(c, launch_gather_acc(c, dc, n_cells, da), "gather launch");
        if (s == HYB_OK && n_cells > 0)
            s = check(c, cudaMemcpyAsync(host_acc + (size_t)k * kMoments * n_cells, da,
                                         8 * (size_t)kMoments * n_cells, cudaMemcpyDeviceToHost, c.stream),
                      "copy moments out");
        if (s == HYB_OK)
            s = check(c, cudaMemcpyAsync(host_status + k, c.st.ctrl + CTRL_STATUS, 4, cudaMemcpyDeviceToHost,
                                         c.stream),
                      "copy status out");
        return s;
    };
    StepHooks hk{copy_in, copy_out};
    hyb_status s = HYB_OK;
    if (!mapped && nsteps == 1) {  // one step: the step's cached graph between the copies
        s = copy_in(0);
        if (s == HYB_OK) s = hyb_hybrid_step(h, dn, n_nodes, dc, n_cells, 1, 1);
        if (s == HYB_OK) s = copy_out(0);
    } else if (!mapped || c.prof_kernel >= 0) {  // pageable buffers or kernel timing: direct launches
        s = copy_in(0);
        if (s == HYB_OK) s = fused_hybrid_steps(c, dn, n_nodes, dc, n_cells, nsteps, &hk);
    } else {
        // the call's graph (transfers and kernels), captured once per steps, parities and buffers
        Ctx::HostKey key;
        key.nsteps = nsteps;
        key.cur_p = c.cur_p;
        key.cur_f = c.cur_f;
        key.nn = n_nodes;
        key.nc = n_cells;
        key.nodes = host_nodes;
        key.cells = host_cells;
        key.acc = host_acc;
        key.status = host_status;
        key.staging = c.io_dev;
        key.dev[0] = mn;
        key.dev[1] = mc;
        key.dev[2] = ma;
        key.dev[3] = ms;
        int slot = -1;
        for (int i = 0; i < 2; ++i)
            if (c.hgraph[i] && c.hkey[i] == key) slot = i;
        if (slot < 0) {
            slot = c.hnext;
            c.hnext ^= 1;
            if (c.hgraph[slot]) {
                cudaGraphExecDestroy(c.hgraph[slot]);
                c.hgraph[slot] = nullptr;
            }
            cudaGraph_t g = nullptr;
            s = check(c, cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            if (s != HYB_OK) return s;
            c.capturing = true;
            hyb_status s2 = copy_in(0);
            if (s2 == HYB_OK) s2 = fused_hybrid_steps(c, dn, n_nodes, dc, n_cells, nsteps, &hk);
            c.capturing = false;
            cudaError_t e = cudaStreamEndCapture(c.stream, &g);
            c.cur_p = key.cur_p;
            c.cur_f = key.cur_f;
            if (s2 != HYB_OK) {
                if (g) cudaGraphDestroy(g);
                return s2;
            }
            s = check(c, e, "end capture");
            if (s != HYB_OK) return s;
            e = cudaGraphInstantiate(&c.hgraph[slot], g, 0);
            cudaGraphDestroy(g);
            s = check(c, e, "graph instantiate");
            if (s != HYB_OK) return s;
            c.hkey[slot] = key;
        }
        s = check(c, cudaGraphLaunch(c.hgraph[slot], c.stream), "graph launch");
        if (s == HYB_OK) {  // each step flips both parities once
            c.cur_p = key.cur_p ^ (nsteps & 1);
            c.cur_f = key.cur_f ^ (nsteps & 1);
        }
    }
    if (s == HYB_OK) s = check(c, cudaEventRecord(c.io_ev[c.io_issued % 4], c.stream), "event record");
    if (s == HYB_OK) c.io_issued += 1;
    return s;
}

hyb_status hyb_host_wait(hyb_ctx* h, int32_t pending) {
    if (!h || pending < 0 || pending > 3) return HYB_EINVAL;
    Ctx& c = h->c;
    while (c.io_issued - c.io_done > pending) {
        hyb_status s = check(c, cudaEventSynchronize(c.io_ev[c.io_done % 4]), "wait for a host step");
        if (s != HYB_OK) return s;
        c.io_done += 1;
    }
    return HYB_OK;
}

void hyb_destroy(hyb_ctx* h) {
    if (!h) return;
    Ctx& c = h->c;
    cudaStreamSynchronize(c.stream);
    drop_graphs(c);
    if (c.io_dev) cudaFree(c.io_dev);
    for (int i = 0; i < 4; ++i)
        if (c.io_ev[i]) cudaEventDestroy(c.io_ev[i]);
    if (c.h_pinned) {
        ProfPool& P = pool_of(c);
        for (size_t i = 0; i < P.a.size(); ++i) {
            cudaEventDestroy(P.a[i]);
            cudaEventDestroy(P.b[i]);
        }
        for (int g = 0; g < 4; ++g)
            if (P.ga[g]) {
                cudaEventDestroy(P.ga[g]);
                cudaEventDestroy(P.gb[g]);
            }
        cudaFreeHost(c.h_pinned);
    }
    delete h;
}

}  // extern "C"
