// The DSMC move of one particle (Sec. 3.1: body-force kick, free flight, fully diffuse
// isothermal walls at x = 0 and x = H, periodic streamwise and spanwise directions) and the
// binning of moved particles into the bins of their new cells. Shared by the DSMC kernels
// and by LB2DSMC, which moves the particles it creates within the fused multi-step pass.
// Compiled without FMA contraction (every translation unit that includes it is), so positions
// and cell keys are the IEEE results of the written expressions.
#pragma once
#include "hyb_internal.cuh"

namespace hyb {

// Particle records (kRec Real each: x, y, vx, vy, vz, z, key bits, unused), read and
// written whole with vector accesses: one 32-byte sector per FP32 record, two per FP64 one.
__device__ __forceinline__ void rec_put(float* rec, int64_t i, float x, float y, float z, float vx,
                                        float vy, float vz, uint32_t tag) {
    float4* p = reinterpret_cast<float4*>(rec + (int64_t)kRec * i);
    p[0] = make_float4(x, y, vx, vy);
    p[1] = make_float4(vz, z, __uint_as_float(tag), 0.0f);
}
__device__ __forceinline__ void rec_put(double* rec, int64_t i, double x, double y, double z, double vx,
                                        double vy, double vz, uint32_t tag) {
    double2* p = reinterpret_cast<double2*>(rec + (int64_t)kRec * i);
    p[0] = make_double2(x, y);
    p[1] = make_double2(vx, vy);
    p[2] = make_double2(vz, z);
    p[3] = make_double2(__longlong_as_double((long long)tag), 0.0);
}
__device__ __forceinline__ void rec_get(const float* rec, int64_t i, float& x, float& y, float& z,
                                        float& vx, float& vy, float& vz, uint32_t& tag) {
    const float4* p = reinterpret_cast<const float4*>(rec + (int64_t)kRec * i);
    const float4 a = p[0], b = p[1];
    x = a.x;
    y = a.y;
    vx = a.z;
    vy = a.w;
    vz = b.x;
    z = b.y;
    tag = __float_as_uint(b.z);
}
__device__ __forceinline__ void rec_get(const double* rec, int64_t i, double& x, double& y, double& z,
                                        double& vx, double& vy, double& vz, uint32_t& tag) {
    const double2* p = reinterpret_cast<const double2*>(rec + (int64_t)kRec * i);
    const double2 a = p[0], b = p[1], c = p[2], d = p[3];
    x = a.x;
    y = a.y;
    vx = b.x;
    vy = b.y;
    vz = c.x;
    z = c.y;
    tag = (uint32_t)__double_as_longlong(d.x);
}
__device__ __forceinline__ uint32_t rec_tag(const float* rec, int64_t i) {
    return __float_as_uint(rec[(int64_t)kRec * i + RS_TAG]);
}
__device__ __forceinline__ uint32_t rec_tag(const double* rec, int64_t i) {
    return (uint32_t)__double_as_longlong(rec[(int64_t)kRec * i + RS_TAG]);
}

// What a move needs: channel sizes, step constants rounded to the state precision, the key.
template <typename Real>
struct MoveCtx {
    Real H, L, Lz;  // channel height (ncx), streamwise period (the channel's rows), spanwise
                    // period (ncz)
    Real dt, g;     // step and body-force velocity increment per step
    int32_t ncx, ncy, ncz;  // the channel's cells; ncz = 0 in 2D
    int32_t y0, nly;        // the rows [y0, y0 + nly) the context holds (0, ncy: all)
    uint32_t bin;           // particle slots per cell
    uint64_t seed;
};

// The cell a particle leaves: its channel cell (the key of its wall draws) and its column,
// channel row and spanwise layer.
struct Origin {
    uint32_t gc;
    int32_t x, y, z;
};

template <typename Real>
__device__ __forceinline__ Origin origin_of(const MoveCtx<Real>& m, uint32_t gc) {
    Origin o;
    o.gc = gc;
    const uint32_t r = gc / (uint32_t)m.ncx;
    o.x = (int32_t)(gc - r * (uint32_t)m.ncx);
    o.y = (int32_t)(r % (uint32_t)m.ncy);
    o.z = (int32_t)(r / (uint32_t)m.ncy);
    return o;
}

// The particles of a cell are ordered, before its collide, by a key their move gives them. A
// particle whose displacement (dx, dy, dz) from its old cell to its new one is at most one
// cell along every axis (the channel and spanwise directions periodic, dy = +1 and -1 the
// same cell in a channel of two rows) gets o bin + k, with o = (3 (dz + 1) + dy + 1) 3 + dx + 1
// (dz = 0 in 2D, o < 9) and k its rank in its old cell; any other particle bit 31 and its
// origin slot, old cell bin + k, so it follows the near ones. Keys are distinct within a cell.
template <typename Real, bool Z3>
__device__ __forceinline__ uint32_t order_key(const MoveCtx<Real>& m, const Origin& o, uint32_t k, int ix,
                                              int iy, int iz) {
    const int dx = ix - o.x;
    int ey = iy - o.y;
    if (ey < 0) ey += m.ncy;
    const int dy = ey == 0 ? 0 : (ey == 1 ? 1 : (ey == m.ncy - 1 ? -1 : 2));
    int dz = 0;
    if constexpr (Z3) {
        int ez = iz - o.z;
        if (ez < 0) ez += m.ncz;
        dz = ez == 0 ? 0 : (ez == 1 ? 1 : (ez == m.ncz - 1 ? -1 : 2));
    }
    if (dx < -1 || dx > 1 || dy > 1 || dz > 1) return 0x80000000u | (o.gc * m.bin + k);
    const int off = (Z3 ? 9 * (dz + 1) : 0) + 3 * (dy + 1) + (dx + 1);
    return (uint32_t)off * m.bin + k;
}

// Diffuse isothermal re-emission from a wall at rest: normal speed sqrt(-2 ln U) into the
// gas, tangential components Gaussian, keyed by (cell, step, rank in cell, bounce).
template <typename Real>
__device__ __forceinline__ void reemit(uint64_t seed, uint32_t cell, uint32_t rank, uint32_t s,
                                       int bounce, Real sign, Real& ux, Real& uy, Real& uz) {
    const uint4 r = draw(seed, cell, s, TAG_WALL, (rank << 3) | (uint32_t)bounce, 0);
    const Real vn = wall_speed<Real>(r.x);
    Real t1, t2;
    gauss_pair<Real>(r.y, r.z, t1, t2);
    ux = sign * vn;
    uy = t1;
    uz = t2;
}

// Flight of a particle whose straight flight crosses a wall: it is re-emitted from the wall
// (diffuse, isothermal), possibly more than once, for the rest of the step.
template <typename Real, bool Z3>
__device__ __forceinline__ void wall_flight(uint64_t seed, uint32_t c, uint32_t k, uint32_t s, Real H,
                                            Real dt, Real& px, Real& py, Real& ux, Real& uy,
                                            Real& uz, uint32_t& hits, uint32_t& caps, Real& pz) {
    Real t = dt;
    for (int b = 0;; ++b) {
        const Real xn = px + ux * t;
        const bool left = xn < (Real)0;
        const bool right = xn > H;
        if (!left && !right) {
            px = xn;
            py = py + uy * t;
            if constexpr (Z3) pz = pz + uz * t;
            break;
        }
        if (b == kMaxBounces) {
            caps += 1;
            px = left ? (Real)0 : H;
            py = py + uy * t;
            if constexpr (Z3) pz = pz + uz * t;
            break;
        }
        hits += 1;
        const Real th = left ? px / (-ux) : (H - px) / ux;
        py = py + uy * th;
        if constexpr (Z3) pz = pz + uz * th;
        px = left ? (Real)0 : H;
        t = t - th;
        if (t < (Real)0) t = (Real)0;
        reemit(seed, c, k, s, b, left ? (Real)1 : (Real)-1, ux, uy, uz);
    }
}

// Periodic wrap of v into [0, period).
template <typename Real>
__device__ __forceinline__ Real wrap_periodic(Real v, Real period) {
    if (v < (Real)0 || v >= period) {
        v = v - period * floor(v / period);
        if (v < (Real)0) v = v + period;
        if (v >= period) v = v - period;
    }
    return v;
}

// Kick (v_y += g), then the flight of one step from (px, py, pz) with walls and periodic
// wrap; the particle is rank k of the channel's cell o at the start of step s (the key of its
// wall draws). Returns its new cell of the context, (iz nly + iy - y0) ncx + ix, with dir = -1;
// for a particle that leaves a streamwise slab, the channel's cell (iz ncy + iy) ncx + ix and
// dir = 0 (towards lower rows) or 1 (higher rows, across the periodic end included). `key` is
// its order key in the new cell.
template <typename Real, bool Z3>
__device__ __forceinline__ uint32_t move_particle(const MoveCtx<Real>& m, const Origin& o, uint32_t k,
                                                  uint32_t s, Real& px, Real& py, Real& pz, Real& ux,
                                                  Real& uy, Real& uz, uint32_t& hits, uint32_t& caps,
                                                  int& dir, uint32_t& key) {
    const uint32_t c = o.gc;
    uy = uy + m.g;
    const Real xn = px + ux * m.dt;
    if (xn >= (Real)0 && xn <= m.H) {
        px = xn;
        py = py + uy * m.dt;
        if constexpr (Z3) pz = pz + uz * m.dt;
    } else {
        wall_flight<Real, Z3>(m.seed, c, k, s, m.H, m.dt, px, py, ux, uy, uz, hits, caps, pz);
    }
    py = wrap_periodic(py, m.L);
    int ix = (int)floor(px), iy = (int)floor(py);
    ix = ix < 0 ? 0 : (ix > m.ncx - 1 ? m.ncx - 1 : ix);
    iy = iy < 0 ? 0 : (iy > m.ncy - 1 ? m.ncy - 1 : iy);
    int iz = 0;
    if constexpr (Z3) {
        pz = wrap_periodic(pz, m.Lz);
        iz = (int)floor(pz);
        iz = iz < 0 ? 0 : (iz > m.ncz - 1 ? m.ncz - 1 : iz);
    }
    key = order_key<Real, Z3>(m, o, k, ix, iy, iz);
    const int iyl = iy - m.y0;
    if (iyl >= 0 && iyl < m.nly) {
        dir = -1;
        return (uint32_t)((iz * m.nly + iyl) * m.ncx + ix);
    }
    // rows above the slab's top and below its bottom, periodically; the nearer side
    const int above = ((iy - (m.y0 + m.nly)) % m.ncy + m.ncy) % m.ncy;
    const int below = ((m.y0 - 1 - iy) % m.ncy + m.ncy) % m.ncy;
    dir = above <= below ? 1 : 0;
    return (uint32_t)((iz * m.ncy + iy) * m.ncx + ix);
}

// A particle that leaves a streamwise slab: appended to the send buffer of its direction
// with its channel cell (counted as lost when the buffer is full).
template <typename Real, bool Z3>
__device__ __forceinline__ void send_particle(Real* const (&xrec)[2], uint32_t* const (&xkey)[2],
                                              uint32_t* const (&xcount)[2], int32_t xcap, int dir,
                                              uint32_t gkey, uint32_t tag, Real px, Real py, Real pz,
                                              Real ux, Real uy, Real uz, uint32_t& lost) {
    const uint32_t slot = atomicAdd(xcount[dir], 1u);
    if (slot < (uint32_t)xcap) {
        rec_put(xrec[dir], slot, px, py, Z3 ? pz : (Real)0, ux, uy, uz, tag);
        xkey[dir][slot] = gkey;
    } else {
        lost += 1;
    }
}

// Appends the active lanes' particles to the bins of their new cells: lanes bound for the
// same cell share one atomic on its count, and each gets arrival = base + rank among them.
// Every lane of the warp calls it (inactive lanes match among themselves under a key no cell
// has). Two particles per lane, both atomics in flight before either result is used.
__device__ __forceinline__ void bin_arrival2(uint32_t* __restrict__ count, uint32_t key1, bool act1,
                                             uint32_t key2, bool act2, unsigned lane, uint32_t& arr1,
                                             uint32_t& arr2) {
    const unsigned peers1 = __match_any_sync(kFull, act1 ? key1 : 0xFFFFFFFFu);
    const unsigned peers2 = __match_any_sync(kFull, act2 ? key2 : 0xFFFFFFFFu);
    const int lead1 = __ffs(peers1) - 1, lead2 = __ffs(peers2) - 1;
    uint32_t b1 = 0, b2 = 0;
    if (act1 && (int)lane == lead1) b1 = atomicAdd(&count[key1], (uint32_t)__popc(peers1));
    if (act2 && (int)lane == lead2) b2 = atomicAdd(&count[key2], (uint32_t)__popc(peers2));
    b1 = __shfl_sync(kFull, b1, lead1);
    b2 = __shfl_sync(kFull, b2, lead2);
    const unsigned below = (1u << lane) - 1u;
    arr1 = b1 + (uint32_t)__popc(peers1 & below);
    arr2 = b2 + (uint32_t)__popc(peers2 & below);
}

// One particle per lane.
__device__ __forceinline__ uint32_t bin_arrival1(uint32_t* __restrict__ count, uint32_t key, bool act,
                                                 unsigned lane) {
    const unsigned peers = __match_any_sync(kFull, act ? key : 0xFFFFFFFFu);
    const int lead = __ffs(peers) - 1;
    uint32_t b = 0;
    if (act && (int)lane == lead) b = atomicAdd(&count[key], (uint32_t)__popc(peers));
    b = __shfl_sync(kFull, b, lead);
    return b + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// One particle half as the move writes it: a moved particle goes to record cell bin +
// arrival, with its order key.
template <typename Real>
struct Half {
    Real* rec;
    uint32_t* count;
};

template <typename Real, bool Z3>
__device__ __forceinline__ void put_particle(const Half<Real>& h, int64_t slot, uint32_t tag, Real px,
                                             Real py, Real pz, Real ux, Real uy, Real uz) {
    rec_put(h.rec, slot, px, py, Z3 ? pz : (Real)0, ux, uy, uz, tag);
}

// Event counters and status of a warp's moves: wall hits, bounce caps and bin overflows.
__device__ __forceinline__ void move_events(unsigned long long* counters, uint32_t* ctrl, uint32_t hits,
                                            uint32_t caps, uint32_t lost, unsigned lane) {
    if (__any_sync(kFull, (hits | caps | lost) != 0u)) {
        hits = __reduce_add_sync(kFull, hits);
        caps = __reduce_add_sync(kFull, caps);
        lost = __reduce_add_sync(kFull, lost);
        if (lane == 0) {
            if (hits) atomicAdd(&counters[HYB_C_WALL_HITS], (unsigned long long)hits);
            if (caps) {
                atomicAdd(&counters[HYB_C_BOUNCE_CAP], (unsigned long long)caps);
                atomicOr(&ctrl[CTRL_STATUS], HYB_ST_BOUNCE_CAP);
            }
            if (lost) atomicOr(&ctrl[CTRL_STATUS], HYB_ST_CAPACITY);
        }
    }
}

}  // namespace hyb
