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
constexpr int kScanTile = 4096;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum CtrlWord {
    CTRL_STATUS = 0,
    CTRL_NTOT = 1,
    CTRL_STEP = 2,
    CTRL_NSAMPLES = 3,
    CTRL_L2D_BASE = 4,
    CTRL_L2D_SKIP = 5,
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
    K_TILE_SUMS = 1,
    K_SCAN = 2,
    K_RANK = 3,
    K_COLLIDE = 4,
    K_LBM = 5,
    K_D2L = 6,
    K_L2D_PREP = 7,
    K_L2D_SAMPLE = 8,
    K_COUNT = 9,
};

// LB2DSMC per-cell record (map_scratch).
struct GradRec {
    double rho;
    double u[3];
    double a2[6];   // packed xx xy xz yy yz zz
    double a3[10];  // packed xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    double C;
    uint32_t nnew;
    uint32_t offset;
};

// Pointers into the arena, resolved for the current ping-pong halves.
struct State {
    void* px[2];
    void* py[2];
    void* pvx[2];
    void* pvy[2];
    void* pvz[2];
    uint32_t* key;
    uint32_t* arrival;
    uint32_t* perm;
    uint32_t* count;
    uint32_t* cell_start;
    uint32_t* tile_sum;
    void* crmax;
    double* rem;
    double* nbar_sum;
    double* acc;
    void* f[2];
    uint32_t* ctrl;
    unsigned long long* counters;
    GradRec* grad;
};

// Everything a kernel needs, passed by value. Particle/population pointers are typed at
// launch.
template <typename Real>
struct DsmcArgs {
    const Real* sx;
    const Real* sy;
    const Real* svx;
    const Real* svy;
    const Real* svz;
    Real* mx;  // in-place move writes into the source half
    Real* my;
    Real* mvx;
    Real* mvy;
    Real* mvz;
    Real* dx;
    Real* dy;
    Real* dvx;
    Real* dvy;
    Real* dvz;
    uint32_t* key;
    uint32_t* arrival;
    uint32_t* perm;
    uint32_t* count;
    uint32_t* cell_start;
    uint32_t* tile_sum;
    Real* crmax;
    double* rem;
    double* nbar_sum;
    double* acc;
    uint32_t* ctrl;
    unsigned long long* counters;
    int32_t ncx, ncy, ncells, ntiles, sample_every, ppc;
    int64_t capacity;
    double dt, g_step, coll_dt, crmax_init;
    uint64_t seed;
};

template <typename Real>
struct LbmArgs {
    const Real* src;
    Real* dst;
    int32_t nx, ny;
    int64_t nnodes;
    double tau, g_step;
};

template <typename Real>
struct MapArgs {
    Real* f;  // current populations
    int32_t nx, ny, ncx, ncy, lb_ratio, ppc, n;
    int64_t nnodes, capacity;
    const int32_t* list;
    double r_lat;
    uint64_t seed;
    const double* acc;
    uint32_t* ctrl;
    unsigned long long* counters;
    GradRec* grad;
    const uint32_t* cell_start;
    Real* x;
    Real* y;
    Real* vx;
    Real* vy;
    Real* vz;
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

// Box-Muller pair in double (the transform Table 1 step 4 names).
__device__ __forceinline__ void box_muller(uint32_t r1, uint32_t r2, double& n1, double& n2) {
    const double rad = sqrt(-2.0 * log(u01open(r1)));
    const double th = 6.283185307179586 * u01open(r2);
    n1 = rad * cos(th);
    n2 = rad * sin(th);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

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
cudaError_t launch_dsmc_step(Ctx& c);
cudaError_t launch_lbm_step(Ctx& c);
cudaError_t launch_map_d2l(Ctx& c, const int32_t* nodes, int32_t n);
cudaError_t launch_map_l2d(Ctx& c, const int32_t* cells, int32_t n);
cudaError_t launch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                                cudaStream_t s);

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
    const int32_t* g_nodes = nullptr;
    const int32_t* g_cells = nullptr;
    int32_t g_nn = -1, g_nc = -1;
    int g_prof = -2;
    int g_curf[2] = {0, 0};        // population parity each graph variant was captured with
    uint32_t* h_pinned = nullptr;  // pinned host words for status reads
};

// Bracket a launch with the timing events when kernel `k` is being profiled.
void prof_begin(Ctx& c, int k);
void prof_end(Ctx& c, int k);

}  // namespace hyb

struct hyb_ctx {
    hyb::Ctx c;
};
