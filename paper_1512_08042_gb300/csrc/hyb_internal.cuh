// Internal definitions of the DSMC-LBM library: context, kernel argument blocks, device
// helpers (Philox4x32-10, uniforms, Box-Muller, Hermite series on packed tensors) and the
// lattice tables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dsmclbm.h"

namespace hyb {

constexpr uint32_t kDeadKey = 0xFFFFFFFFu;
constexpr int kMoments = 20;
constexpr int kMaxBounces = 8;
constexpr int kMaxScatterBlocks = 16;
constexpr int kMaxL2DAttempts = 1000;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum CtrlWord {
    CTRL_STATUS = 0,
    CTRL_NTOT = 1,
    CTRL_STEP = 2,
    CTRL_NSAMPLES = 3,
    CTRL_RESERVED4 = 4,
    CTRL_NACC = 5,     // particles counted by the collide pass in progress
    CTRL_WORDS = 16,
};

enum Tag : uint32_t {
    TAG_INIT_POS = 1,
    TAG_INIT_VEL = 2,
    TAG_WALL = 3,
    TAG_NTC_PAIR = 4,
    TAG_NTC_SCAT = 5,
    TAG_L2D_VEL = 6,
    TAG_L2D_POS = 7,
    TAG_L2D_ROUND = 8,
};

enum KernelId {
    K_MOVE = 0,
    K_COLLIDE = 1,
    K_LBM = 2,
    K_D2L = 3,
    K_L2D = 4,
    K_FUSED = 5,  // the fused collide-and-move pass of multi-step calls
    K_COUNT = 6,
};

// LB2DSMC per-cell record (map_scratch): the Grad record of one coupling cell (176 bytes),
// FP64: rho, the new particle count and v = a2[6] (xx xy xz yy yz zz), a3[10] (xxx xxy xxz
// xyy xyz xzz yyy yyz yzz zzz), u[3], C.
struct GradRec {
    double rho;
    uint32_t nnew;
    uint32_t pad;
    double v[20];
};
enum : int { GR_A2 = 0, GR_A3 = 6, GR_U = 16, GR_C = 19 };

// A particle is one record of kRec Real values: x, y, vx, vy, vz, z (3D only), its
// order key (the bits of a u32, written by the move) and one unused value, so that in
// FP32 one record fills one 32-byte sector and a scattered write of a moved particle writes
// whole sectors.
constexpr int kRec = 8;
enum RecSlot : int { RS_X = 0, RS_Y = 1, RS_VX = 2, RS_VY = 3, RS_VZ = 4, RS_Z = 5, RS_TAG = 6 };

// Pointers into the arena.
struct State {
    void* part[2];  // particle records, Real[capacity][kRec]
    uint32_t* count[2];
    uint8_t* coupled;  // per cell: 1 while a fused multi-step call regenerates the cell
    char* xsend[2];    // a slab's exchange buffers (count, records, cell ids)
    char* xrecv[2];
    void* crmax;
    void* rem;
    uint32_t* nbar_sum;
    double* acc;
    void* f[2];
    uint32_t* ctrl;
    unsigned long long* counters;
    GradRec* grad;
    void* coll_cell;  // per-cell NTC factor (Kn profile), or null
    void* tau_node;   // per-node relaxation time (Kn profile), or null
};

// Everything a DSMC kernel needs, passed by value, for a step that starts from the sorted
// particles of half p (srec): the move appends each particle, with its order key, to the
// bin of its new cell in half p^1 (drec); the collide puts each cell
// of half p^1 in stable order in place, collides and samples it; the fused pass takes the
// arrivals of half p^1 through the collide and moves them on into half p for the next step.
template <typename Real>
struct DsmcArgs {
    Real* srec;  // particle records of half p
    Real* drec;  // particle records of half p^1
    uint32_t* count_s;
    uint32_t* count_d;
    Real* crmax;
    Real* rem;
    uint32_t* nbar_sum;
    double* acc;
    uint32_t* ctrl;
    unsigned long long* counters;
    const uint8_t* coupled;  // cells regenerated by the step's LB2DSMC (fused pass), or null
    int32_t ncx, ncy, ncells, bin, sample_every, ppc;
    double dt, g_step, coll_dt, crmax_init;
    // dt, g_step and coll_dt rounded to the state precision on the host (the kernels take
    // no FP64 conversion per cell)
    Real dt_r, g_r, coll_r;
    const Real* coll_cell;  // per-cell NTC factor, or null for coll_dt everywhere
    uint64_t seed;
    int32_t ncz;  // 3D (ncz >= 2): cells along z; 0 in 2D
    // a streamwise slab: its first row in the channel and the channel's rows (0 and ncy for
    // the whole channel); its exchange buffers: send records towards lower (0) and higher (1)
    // rows with the particles' channel cells and counts, and the records received from the
    // slab below (0) and above (1)
    int32_t y0, ncy_g;
    int32_t xcap;
    Real* xrec[2];
    uint32_t* xkey[2];
    uint32_t* xcount[2];
    const Real* rrec[2];
    const uint32_t* rkey[2];
    const uint32_t* rcount[2];
};

template <typename Real>
struct LbmArgs {
    const Real* src;
    Real* dst;
    int32_t nx, ny;
    int64_t nnodes;
    Real om, of, g_step;  // 1 - 1/tau, 1 - 1/(2 tau), force increment per step
    // per-node force increment and relaxation time (differentiated LBM); unused by the
    // plain step
    const Real* g_node;
    const Real* tau_node;
    int32_t bgk;  // 1: unregularised BGK collision (lb_collision)
    int32_t nz;   // lattice layers along z (1 in 2D)
};

// One step of the adjoint of the LBM with per-node parameters: lam_next = dL/df_{t+1} in,
// lam = dL/df_t out, the parameter gradients accumulated; wall = 2 ny adjoint wall
// densities (left rows, then right rows) followed by a 32-bit block ticket, all zero on entry
// and left zero.
template <typename Real>
struct LbmAdjArgs {
    const Real* f;         // populations at t
    const Real* lam_next;  // adjoint at t + 1
    Real* lam;             // adjoint at t
    const Real* g_node;
    const Real* tau_node;
    Real* grad_g;
    Real* grad_tau;
    Real* wall;  // 2 nrows wall sums (left, right; row z ny + y) and a ticket
    int32_t nx, ny, nz;
    int64_t nnodes;
};

template <typename Real>
struct MapArgs {
    Real* f;  // current populations
    int32_t nx, ny, ncx, ncy, lb_ratio, ppc, n, bin;
    int64_t nnodes;
    const int32_t* list;
    int32_t eq_mode;  // DSMC2LB: 1 the local equilibrium of rho, u only (d2l_mode)
    double r_lat;
    uint64_t seed;
    const double* acc;
    uint32_t* ctrl;
    unsigned long long* counters;
    GradRec* grad;
    uint32_t* count;  // current half
    Real* rec;        // particle records of the current half
    int32_t ncz;      // 3D (ncz >= 2): cells along z; 0 in 2D
    // fused multi-step pass (LB2DSMC that moves what it creates): the half that receives the
    // next step's arrivals and its counts, and the move's step constants
    Real* arec;
    uint32_t* acount;
    Real dt_r, g_r;
    // a streamwise slab: its first row in the channel and the channel's rows (cell ids of the
    // random streams and y positions are the channel's) and the ghost rows below its LB rows
    int32_t y0, ncy_g, yh;
};

// ---------------------------------------------------------------------------------------
// Device helpers

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t entity, uint32_t step, uint32_t tag,
                                      uint32_t sub, uint32_t block) {
    return philox(make_uint4(entity, step, (tag << 24) | (sub & 0xFFFFFFu), block), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float u01f(uint32_t r) { return (float)(r >> 8) * 0x1p-24f; }
__device__ __forceinline__ double u01open(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }
__device__ __forceinline__ double u01d(uint32_t r) { return (double)r * 0x1p-32; }
__device__ __forceinline__ uint32_t uindex(uint32_t r, uint32_t n) {
    return (uint32_t)(((uint64_t)r * n) >> 32);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// The channel's id of cell c = (iz nly + iy) ncx + ix of a streamwise slab whose rows start
// at row y0 of a channel of ncy_g rows: (iz ncy_g + y0 + iy) ncx + ix (c itself for the whole
// channel, y0 = 0 and nly = ncy_g).
__host__ __device__ __forceinline__ uint32_t global_cell(uint32_t c, int ncx, int nly, int y0,
                                                          int ncy_g) {
    if (y0 == 0 && nly == ncy_g) return c;
    const uint32_t plane = (uint32_t)ncx * (uint32_t)nly;
    const uint32_t iz = c / plane, r = c - iz * plane;
    return (iz * (uint32_t)ncy_g + (uint32_t)y0) * (uint32_t)ncx + r;
}

// Kernel arguments of one context, or of a batch of independent contexts (replicas). The
// units of a launch (cells, blocks of cells, nodes or list entries) are numbered across the
// replicas: unit u belongs to replica r with pre[r] <= u < pre[r + 1] and is unit u - pre[r]
// of that replica. Kernels are instantiated for both cases; a single context takes its
// arguments from the launch parameters and pays nothing for the batch form.
template <class Args>
struct Launch {
    Args one;             // the context's arguments (single form)
    const Args* tab;      // per-replica arguments in device memory (batch form)
    const int64_t* pre;   // nrep + 1 prefix sums of the units per replica (batch form)
    int32_t nrep;
    int64_t total;        // units of the launch
};

__device__ __forceinline__ int replica_of(const int64_t* pre, int nrep, int64_t u) {
    int lo = 0, hi = nrep;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Programmatic dependent launch (sm_90 and later). The kernels of a step are launched with
// launch_pdl: each one first lets the next kernel of the stream be scheduled
// (launch_dependents), then waits until the previous kernel has completed and its writes are
// visible (wait). The launch latency and block ramp-up of a kernel so overlap the tail of
// the one before it; no work that reads the previous kernel's results comes before the wait.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Asynchronous 16-byte copies from global to shared memory (cp.async, sm_80 and later),
// committed as one group; wait_all waits for all of the thread's groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Float elementary functions of the FP32 state path, evaluated from their series with every
// operation fixed (this code is compiled without FMA contraction), so that the results are
// reproducible bit for bit:
//   ln x = e ln 2 + 2 atanh(s), x = m 2^e, m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
//          atanh by its odd series to s^11 (Abramowitz & Stegun 4.6.22);
//   sin, cos (2 pi u), u in [0,1) with 24 bits: exact reduction of 4u to a quadrant and of
//          the remainder to [0, 1/2], then the Taylor series of sin and cos on [0, pi/4]
//          (A&S 4.3.65, 4.3.66).
__device__ __forceinline__ float ln_f(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e += 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float t = 1.0f / 11.0f;
    t = t * s2 + 1.0f / 9.0f;
    t = t * s2 + 1.0f / 7.0f;
    t = t * s2 + 1.0f / 5.0f;
    t = t * s2 + 1.0f / 3.0f;
    t = t * s2 + 1.0f;
    const float lnm = 2.0f * s * t;
    const float fe = (float)e;
    return fe * 0.693145751953125f + (fe * 1.4286068203e-06f + lnm);
}

__device__ __forceinline__ void sincos2pi_f(float u, float& sn, float& cs) {
    const float t = 4.0f * u;
    const float k = floorf(t);
    const float f = t - k;
    const int q = (int)k & 3;
    const bool swap = f > 0.5f;
    const float g = swap ? 1.0f - f : f;
    const float phi = g * 1.57079637f;
    const float p2 = phi * phi;
    float ps = 1.0f / 362880.0f;
    ps = ps * p2 - 1.0f / 5040.0f;
    ps = ps * p2 + 1.0f / 120.0f;
    ps = ps * p2 - 1.0f / 6.0f;
    ps = ps * p2 + 1.0f;
    const float sp = phi * ps;
    float pc = -1.0f / 3628800.0f;
    pc = pc * p2 + 1.0f / 40320.0f;
    pc = pc * p2 - 1.0f / 720.0f;
    pc = pc * p2 + 1.0f / 24.0f;
    pc = pc * p2 - 0.5f;
    pc = pc * p2 + 1.0f;
    const float sa = swap ? pc : sp;
    const float ca = swap ? sp : pc;
    if (q == 0) {
        sn = sa;
        cs = ca;
    } else if (q == 1) {
        sn = ca;
        cs = -sa;
    } else if (q == 2) {
        sn = -sa;
        cs = -ca;
    } else {
        sn = -ca;
        cs = sa;
    }
}

// Unit normal pair (Box-Muller) and diffuse-wall normal speed sqrt(-2 ln U) in the state
// precision: float uses 24-bit uniforms (U1 in (0,1]) and the series above; double uses the
// double library functions with 32-bit uniforms.
template <typename Real>
__device__ __forceinline__ void gauss_pair(uint32_t r1, uint32_t r2, Real& n1, Real& n2);
template <>
__device__ __forceinline__ void gauss_pair<float>(uint32_t r1, uint32_t r2, float& n1, float& n2) {
    const float u1 = (float)((r1 >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(r2 >> 8) * 0x1p-24f;
    const float rad = sqrtf(-2.0f * ln_f(u1));
    float sn, cs;
    sincos2pi_f(u2, sn, cs);
    n1 = rad * cs;
    n2 = rad * sn;
}
template <>
__device__ __forceinline__ void gauss_pair<double>(uint32_t r1, uint32_t r2, double& n1, double& n2) {
    const double rad = sqrt(-2.0 * log(u01open(r1)));
    const double th = 6.283185307179586 * u01open(r2);
    n1 = rad * cos(th);
    n2 = rad * sin(th);
}
template <typename Real>
__device__ __forceinline__ Real wall_speed(uint32_t r);
template <>
__device__ __forceinline__ float wall_speed<float>(uint32_t r) {
    const float u = (float)((r >> 8) + 1u) * 0x1p-24f;
    return sqrtf(-2.0f * ln_f(u));
}
template <>
__device__ __forceinline__ double wall_speed<double>(uint32_t r) {
    return sqrt(-2.0 * log(u01open(r)));
}

// Packed symmetric tensors: rank 2 order xx xy xz yy yz zz, rank 3 order xxx xxy xxz xyy
// xyz xzz yyy yyz yzz zzz. Full contractions weight each packed entry by its number of
// index permutations.
__device__ __forceinline__ double herm2_contract(const double* a2, const double* x) {
    // sum_ij a_ij (x_i x_j - d_ij)
    return a2[0] * (x[0] * x[0] - 1.0) + a2[3] * (x[1] * x[1] - 1.0) + a2[5] * (x[2] * x[2] - 1.0) +
           2.0 * (a2[1] * x[0] * x[1] + a2[2] * x[0] * x[2] + a2[4] * x[1] * x[2]);
}

__device__ __forceinline__ double herm3_contract(const double* a3, const double* x) {
    // sum_ijk a_ijk (x_i x_j x_k - x_i d_jk - x_j d_ik - x_k d_ij)
    const double X = x[0], Y = x[1], Z = x[2];
    const double cubic = a3[0] * X * X * X + 3.0 * a3[1] * X * X * Y + 3.0 * a3[2] * X * X * Z +
                         3.0 * a3[3] * X * Y * Y + 6.0 * a3[4] * X * Y * Z +
                         3.0 * a3[5] * X * Z * Z + a3[6] * Y * Y * Y + 3.0 * a3[7] * Y * Y * Z +
                         3.0 * a3[8] * Y * Z * Z + a3[9] * Z * Z * Z;
    // trace vector t_i = sum_j a_ijj
    const double tx = a3[0] + a3[3] + a3[5];
    const double ty = a3[1] + a3[6] + a3[8];
    const double tz = a3[2] + a3[7] + a3[9];
    return cubic - 3.0 * (tx * X + ty * Y + tz * Z);
}

// ---------------------------------------------------------------------------------------
// Lattices (Shan, Yuan, Chen 2006 Gauss-Hermite sets). Row order is the population layout.
struct D3Q39 {
    static constexpr int Q = 39;
    static constexpr int ORDER = 3;
    static constexpr int MAXV = 3;
};
struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int ORDER = 2;
    static constexpr int MAXV = 1;
};

template <class LAT>
struct LatTab;

// The tables are local constants of __host__ __device__ constexpr functions, so device code
// may index them at run time as well as fold them at compile time.
template <>
struct LatTab<D3Q39> {
    __host__ __device__ static constexpr int e(int a, int i) {
        constexpr int t[39][3] = {
            {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
            {1, 1, 1},   {-1, 1, 1},  {1, -1, 1},  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1},
            {-1, -1, -1}, {2, 0, 0},  {-2, 0, 0},  {0, 2, 0},   {0, -2, 0},  {0, 0, 2},  {0, 0, -2},
            {2, 2, 0},   {-2, 2, 0},  {2, -2, 0},  {-2, -2, 0}, {2, 0, 2},   {-2, 0, 2}, {2, 0, -2},
            {-2, 0, -2}, {0, 2, 2},   {0, -2, 2},  {0, 2, -2},  {0, -2, -2}, {3, 0, 0},  {-3, 0, 0},
            {0, 3, 0},   {0, -3, 0},  {0, 0, 3},   {0, 0, -3}};
        return t[a][i];
    }
    __host__ __device__ static constexpr double w(int a) {
        return a == 0 ? 1.0 / 12.0
               : a <= 6 ? 1.0 / 12.0
               : a <= 14 ? 1.0 / 27.0
               : a <= 20 ? 2.0 / 135.0
               : a <= 32 ? 1.0 / 432.0
                         : 1.0 / 1620.0;
    }
};

template <>
struct LatTab<D3Q19> {
    __host__ __device__ static constexpr int e(int a, int i) {
        constexpr int t[19][3] = {
            {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
            {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1}, {1, 0, -1},
            {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
        return t[a][i];
    }
    __host__ __device__ static constexpr double w(int a) {
        return a == 0 ? 1.0 / 3.0 : a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0;
    }
};

template <class LAT>
__host__ __device__ constexpr double lat_r() {
    return LAT::Q == 39 ? 1.2247448713915889 : 1.7320508075688772;
}

// Sum over populations entering through a wall of e_x * w_a (mass flux of the wall
// Maxwellian per unit density).
template <class LAT>
__host__ __device__ constexpr double wall_flux_norm() {
    double s = 0.0;
    for (int a = 0; a < LAT::Q; ++a)
        if (LatTab<LAT>::e(a, 0) > 0) s += LatTab<LAT>::e(a, 0) * LatTab<LAT>::w(a);
    return s;
}

// ---------------------------------------------------------------------------------------
// Launchers (defined in the kernel translation units).
struct Ctx;
cudaError_t launch_init(Ctx& c);
cudaError_t launch_dsmc_step(Ctx& c);  // move and collide of one step from half cur_p
// The passes of a DSMC step from half p (DsmcArgs of parity p): the move (p -> p^1), the
// collide (p^1 in place) and the fused pass (collide p^1, then move into p).
cudaError_t launch_dsmc_move(Ctx& c, int p);
cudaError_t launch_dsmc_collide(Ctx& c, int p);
cudaError_t launch_dsmc_fused(Ctx& c, int p);
bool dsmc_fused_fills_gpu(const Ctx& c);
// A streamwise slab: appends the received particles to the bins of half p^1 after the move.
cudaError_t launch_dsmc_merge(Ctx& c, int p);
// Marks (v = 1) or clears (v = 0) the listed cells in the coupled-cell mask.
cudaError_t launch_mark_cells(Ctx& c, const int32_t* cells, int32_t n, uint8_t v);
cudaError_t launch_lbm_step(Ctx& c);
// A streamwise slab's LB ghost rows: values per side, and the pack (unpack = 0) or unpack of
// one side's exchanged populations.
int64_t lbm_halo_values(const Ctx& c);
cudaError_t launch_lbm_halo(Ctx& c, int side, void* buf, int unpack);
cudaError_t launch_lbm_step_nodes(Ctx& c, const void* f_src, void* f_dst, const void* g, const void* tau);
cudaError_t launch_lbm_adjoint_step(Ctx& c, const void* f, const void* lam_next, void* lam,
                                    const void* g, const void* tau, void* grad_g, void* grad_tau,
                                    void* wall);
cudaError_t launch_interface_loss(Ctx& c, const void* f, const int32_t* nodes, int32_t n,
                                  const void* targets, double* loss, void* lam);
cudaError_t launch_map_d2l(Ctx& c, const int32_t* nodes, int32_t n);
cudaError_t launch_map_l2d(Ctx& c, const int32_t* cells, int32_t n);
cudaError_t launch_map_l2d_noalloc(Ctx& c, const int32_t* cells, int32_t n);
// LB2DSMC within the fused pass: the listed cells' particles are in half p^1 (left there in
// stable order by the fused pass of parity p); the cells are regenerated (or, if the new
// count exceeds the bin, kept) and their particles moved on into half p.
cudaError_t launch_map_l2d_move(Ctx& c, const int32_t* cells, int32_t n, int p);
cudaError_t launch_gather_acc(Ctx& c, const int32_t* cells, int32_t n, double* out);
// Host-buffer steps with page-locked buffers: the lists copied in by a kernel that reads host
// memory, the listed cells' sums and the status word written to host memory by one kernel
// (device-addressable pointers of the host buffers).
cudaError_t launch_lists_in(Ctx& c, const int32_t* hn, int32_t nn, const int32_t* hc, int32_t nc,
                            int32_t* dn, int32_t* dc);
cudaError_t launch_results_out(Ctx& c, const int32_t* cells, int32_t n, double* out,
                               uint32_t* status_out);
cudaError_t launch_map_d2l_adjoint(Ctx& c, const int32_t* nodes, int32_t n, void* lam,
                                   double* grad_acc);
cudaError_t launch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                                cudaStream_t s);

// A batch of independent replicas (hyb_batch in runtime.cu): the per-replica kernel
// arguments of each ping-pong parity and the unit prefix sums, in a table region of the
// batch arena, and the block shapes picked by the tuner.
struct BatchDev {
    int32_t nrep = 0;
    int32_t real_bytes = 4, lattice = 39;
    int32_t lb_collision = 0;  // one collision for all replicas
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    const void* dsmc[2] = {nullptr, nullptr};               // DsmcArgs<Real>[nrep], by particle half
    const void* lbm[2] = {nullptr, nullptr};                // LbmArgs<Real>[nrep], by population half
    const void* d2l[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // MapArgs, [particle][population]
    const void* l2d[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    const int64_t* pre_cells = nullptr;
    const int64_t* pre_blocks = nullptr;   // collide blocks of 32 cells
    const int64_t* pre_blocks4 = nullptr;  // collide blocks of 16 cells
    const int64_t* pre_nodes = nullptr;
    const int64_t* pre_d2l = nullptr;
    const int64_t* pre_l2d = nullptr;
    int64_t tot_cells = 0, tot_blocks = 0, tot_blocks4 = 0, tot_nodes = 0, tot_d2l = 0, tot_l2d = 0;
    // collide shared-memory pools of 32- and 16-cell blocks: the largest over the replicas
    uint32_t pool = 0, pool4 = 0;
    uint32_t maxbin = 0;  // the largest bin over the replicas (the collide's key bitmaps)
    // threads per block of each tuned class (the collide: 256 for 32 cells, 128 for 16)
    int move_block = 256, lbm_block = 128, d2l_block = 128, collide_block = 256;
};
size_t dsmc_args_bytes(int real_bytes);
void dsmc_args_fill(Ctx& c, int cur_p, void* out);
size_t lbm_args_bytes(int real_bytes);
void lbm_args_fill(Ctx& c, int cur_f, void* out);
size_t map_args_bytes(int real_bytes);
void map_args_fill(Ctx& c, int cur_p, int cur_f, const int32_t* list, int32_t n, void* out);
uint32_t collide_pool(const Ctx& c, int warps = 8);
cudaError_t launch_batch_move(BatchDev& b, int cur_p);
cudaError_t launch_batch_collide(BatchDev& b, int cur_p);
cudaError_t launch_batch_lbm(BatchDev& b, int cur_f);
cudaError_t launch_batch_d2l(BatchDev& b, int cur_p, int cur_f);
cudaError_t launch_batch_l2d(BatchDev& b, int cur_p, int cur_f);

// Kernel timing: a pool of event pairs for direct launches, and one fixed pair per graph
// variant (a graph replay records into the pair captured in it).
struct ProfPool {
    std::vector<cudaEvent_t> a, b;
    size_t used = 0;
    cudaEvent_t ga[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t gb[4] = {nullptr, nullptr, nullptr, nullptr};
    bool gpending[4] = {false, false, false, false};
    int capture_slot = 0;
};

// Host context.
struct Ctx {
    hyb_params p;
    hyb_derived d;
    hyb_layout L;
    char* arena = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int cur_p = 0;  // current particle half
    int cur_f = 0;  // current population half
    State st{};
    int num_sms = 152;
    std::string err;
    // kernel timing
    int prof_kernel = -1;
    ProfPool pool;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    bool capturing = false;
    // graphs of one hybrid step, per particle parity
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // graphs of a whole multi-step (fused) hybrid call: two slots keyed by the step count and
    // the parities it starts from
    cudaGraphExec_t mgraph[2] = {nullptr, nullptr};
    int32_t mkey[2][3] = {{-1, -1, -1}, {-1, -1, -1}};
    int mnext = 0;
    // graphs of multi-step host-buffer calls, keyed by steps, parities, lists and buffers
    // (the host buffers by their host and device addresses: a buffer registered again at the
    // same host address may get another device address)
    struct HostKey {
        int32_t nsteps = -1, cur_p = -1, cur_f = -1, nn = -1, nc = -1;
        const void *nodes = nullptr, *cells = nullptr, *acc = nullptr, *status = nullptr, *staging = nullptr;
        const void* dev[4] = {nullptr, nullptr, nullptr, nullptr};
        bool operator==(const HostKey& o) const {
            return nsteps == o.nsteps && cur_p == o.cur_p && cur_f == o.cur_f && nn == o.nn && nc == o.nc &&
                   nodes == o.nodes && cells == o.cells && acc == o.acc && status == o.status &&
                   staging == o.staging && dev[0] == o.dev[0] && dev[1] == o.dev[1] && dev[2] == o.dev[2] &&
                   dev[3] == o.dev[3];
        }
    };
    cudaGraphExec_t hgraph[2] = {nullptr, nullptr};
    HostKey hkey[2];
    int hnext = 0;
    const int32_t* g_nodes = nullptr;
    const int32_t* g_cells = nullptr;
    int32_t g_nn = -1, g_nc = -1;
    int g_prof = -2;
    int g_curf[2] = {0, 0};        // population parity each graph variant was captured with
    uint32_t* h_pinned = nullptr;  // pinned host words for status reads
    bool split_pending = false;    // a slab's dsmc_move was issued, its collide is due
    int fuse_mode = 0;             // HYB_FUSE_*: multi-step calls fuse the DSMC passes
    int fuse_pays = -1;            // HYB_FUSE_AUTO's choice, formed at the first multi-step call
    int collide_warps = 8;         // collide block shape: 8 warps (32 cells) or 4 (16 cells)
    // hyb_hybrid_step_host: device staging of the lists and the gathered moment sums, and a
    // ring of completion events of the steps in flight
    char* io_dev = nullptr;
    size_t io_bytes = 0;
    cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t io_issued = 0, io_done = 0;
};

// Bracket a launch with the timing events when kernel `k` is being profiled.
void prof_begin(Ctx& c, int k);
void prof_end(Ctx& c, int k);

}  // namespace hyb

struct hyb_ctx {
    hyb::Ctx c;
};
