/*
 * dsmclbm.h - C ABI of the GB300 (sm_103a) hot path of the hybrid DSMC-LBM method of
 * Di Staso, Clercx, Succi and Toschi, "DSMC-LBM mapping scheme for rarefied and
 * non-rarefied gas flows" (arXiv 1512.08042).
 *
 * The library advances a force-driven plane channel (Sec. 3.1) with two solvers and maps
 * between them (Sec. 2):
 *   dsmc_step        DSMC of a hard-sphere gas: move with diffuse isothermal walls, binning
 *                    by cell in a fixed order, no-time-counter collisions (Sec. 5,
 *                    Eq. collisionnumber), per-cell Hermite-moment sampling.
 *   lbm_step         regularised BGK lattice Boltzmann on D3Q39 (Hermite order 3) or D3Q19
 *                    (order 2) with kinetic walls and a body force (Sec. 2 "ingredients",
 *                    Sec. 3.1, Eq. tau).
 *   map_dsmc_to_lbm  DSMC2LB projection (Sec. 2.1, Eq. discretefunctions).
 *   map_lbm_to_dsmc  LB2DSMC reconstruction by acceptance-rejection (Sec. 2.2, Table 1).
 *   sample_moments   the cumulative DSMC moment sums the projection reads (Sec. 2.1, Fig. 1).
 *
 * Units: lengths in DSMC cells, velocities in c_th = sqrt(kT/m) (Hermite units, unit-variance
 * weight function of Eq. globalMax), one DSMC step = one LB step = T0 of Appendix A with the
 * isothermal sound speed. LB density 1 corresponds to `ppc` particles per DSMC cell.
 *
 * Memory: the caller owns all device memory. It allocates one arena of
 * hyb_layout.total_bytes (256-byte aligned) on the device and passes it to dsmc_init; the
 * library keeps a borrowed pointer for the context's lifetime and never frees it. Byte
 * offsets of every array inside the arena are given by hyb_layout_compute, so the caller can
 * read and write state directly (e.g. through torch tensors).
 *
 * Streams: every call that launches work enqueues it on the stream given to dsmc_init and
 * returns without synchronising, except the functions marked "synchronises". Argument errors
 * return HYB_EINVAL and launch nothing. Errors found on the device (capacity overflow, a
 * capped device loop, a bad coupling index) are recorded in a sticky status word that
 * hyb_sync_status reads. No C++ exception and no exit() crosses this interface.
 */
#ifndef DSMCLBM_H
#define DSMCLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HYB_ABI_VERSION 12u

typedef enum {
    HYB_OK = 0,
    HYB_EINVAL = 1,     /* invalid argument; nothing was launched */
    HYB_ENOMEM = 2,     /* arena too small */
    HYB_ECUDA = 3,      /* a CUDA runtime call failed; see hyb_last_error */
    HYB_ECAPACITY = 4,  /* particle capacity or per-cell bound exceeded on the device */
    HYB_ETIMEOUT = 5,   /* a capped device loop (wall bounces, scattering draws) hit its cap */
    HYB_ESAMPLING = 6,  /* LB2DSMC acceptance-rejection hit its attempt cap */
    HYB_ESTATE = 7      /* call out of order (e.g. graph capture already in progress) */
} hyb_status;

/* Bits of the sticky device status word. */
#define HYB_ST_CAPACITY (1u << 0)      /* a cell's particles exceeded its bin of slots */
#define HYB_ST_BOUNCE_CAP (1u << 1)    /* a particle hit the walls more than 8 times in a step */
#define HYB_ST_SCATTER_CAP (1u << 2)   /* 32 Marsaglia draws rejected in a row */
#define HYB_ST_SAMPLING_CAP (1u << 3)  /* 1000 LB2DSMC trials rejected in a row */
#define HYB_ST_CELL_OVERFLOW (1u << 4) /* more than 2^24 NTC candidates in one cell */
#define HYB_ST_BAD_INPUT (1u << 5)     /* coupling index out of range, or no DSMC samples */

/* Counters (hyb_read_counters): index meaning. */
#define HYB_C_WALL_HITS 0
#define HYB_C_CANDIDATES 1
#define HYB_C_COLLISIONS 2
#define HYB_C_CREATED 3
#define HYB_C_DELETED 4
#define HYB_C_L2D_ATTEMPTS 5
#define HYB_C_ENVELOPE 6   /* trials with G > C, which the envelope C g0 does not cover */
#define HYB_C_BOUNCE_CAP 7
#define HYB_NCOUNTERS 16

/* Problem parameters (plain data; the library copies it). */
typedef struct {
    uint32_t abi_version;   /* HYB_ABI_VERSION */
    int32_t ncx;            /* DSMC cells across the channel; walls at x = 0 and x = ncx (>= 6) */
    int32_t ncy;            /* DSMC cells streamwise, periodic (>= 1) */
    int32_t lb_ratio;       /* LB nodes per DSMC cell per axis: 1 or 2 */
    int32_t ppc;            /* particles per cell at initialisation (>= 1) */
    int32_t lattice;        /* 39: D3Q39, Hermite order 3; 19: D3Q19, order 2 */
    int32_t real_bytes;     /* 4: float particle and population state; 8: double */
    int32_t sample_every;   /* moments sampled every `sample_every` DSMC steps (>= 1) */
    uint64_t seed;          /* Philox key */
    double kn;              /* Knudsen number on the channel height (> 0) */
    double ma;              /* Mach number of the no-slip centreline velocity, u_max / c_s */
    double crmax_init;      /* initial (sigma_T c_r)_max / sigma_T in c_th units (> 0) */
    double capacity_factor; /* slots per cell: bin = 32 * ceil(capacity_factor * ppc / 32),
                               at most 256 */
    double T_K;             /* temperature [K], for SI conversion only */
    double mass_kg;         /* molecular mass [kg], for SI conversion only */
    int32_t lb_collision;   /* 0: regularised BGK (Sec. 2); 1: plain BGK, f' = f_eq +
                               (1 - 1/tau)(f - f_eq) + (1 - 1/(2 tau)) F, the LB model of the
                               proof-of-concept hybrid (Sec. 4) */
    int32_t d2l_mode;       /* 0: DSMC2LB to the lattice's Hermite order from rho, u, P, Q
                               (Sec. 2.1); 1: the local equilibrium from rho and u only
                               (Sec. 4, Eq. feq_dsmc; to order 3 on D3Q39) */
    int32_t kn_profile;     /* 0: one Kn; 1: Kn varies along the channel, log-linear in the
                               streamwise coordinate y (cell units) from kn at y = 0 to kn_end
                               at y = ncy / 2 and back: Kn(y) = kn (kn_end / kn)^s,
                               s = 1 - |2 y / ncy - 1|. Each DSMC cell takes the NTC factor
                               of Eq. collisionnumber at Kn(iy + 1/2), each LB node the tau
                               of Eq. tau at Kn((j + 1/2) / lb_ratio) (j its row); the body
                               force stays that of kn. Not with a batch. */
    int32_t pad0;
    double kn_end;          /* Kn at y = ncy / 2 when kn_profile = 1 (> 0) */
    int32_t ncz;            /* DSMC cells along z, periodic (the paper's solvers are 3D with
                               periodic y and z, Sec. 3.1): 0 or 1 for the quasi-2D slab of
                               one cell and one LB layer; >= 2 for full 3D, with particle z
                               positions, ncz * lb_ratio LB layers, cells (iz ncy + iy) ncx + ix
                               and nodes (z ny + y) nx + x. Not with a batch. */
    int32_t accum_mode;     /* moment sums: 0 = FP64 cumulative sums (one FP64 addition per sum
                               per step, of that step's cell sum); 1 = Kahan-compensated FP32,
                               not built: HYB_EINVAL */
    int32_t ncy_global;     /* 0: the context holds the whole channel. > 0: the context is one
                               streamwise slab of a channel of ncy_global DSMC rows (periodic):
                               the rows [y0, y0 + ncy) (ncy >= 4), with the channel's ncx, ncz,
                               ppc, Kn, seed and lattice. Cell ids in the random streams and the
                               order keys, and particle y positions, are the channel's, so
                               slabs stepped with the exchange below give the whole channel's
                               results bit for bit. The LB lattice of a slab has yh ghost rows
                               below and above its ncy * lb_ratio rows (hyb_derived.yh), filled
                               from the neighbours by lbm_halo_pack / lbm_halo_unpack before each
                               LB step; particles leaving the slab go to its two send buffers
                               (hyb_layout.xsend: 0 towards lower rows, 1 towards higher), which
                               the caller copies into the neighbours' receive buffers (xrecv: 0
                               from the slab below, 1 from the slab above) before dsmc_merge.
                               A slab is advanced with dsmc_move, dsmc_merge, dsmc_collide and
                               lbm_step; dsmc_step and hyb_hybrid_step return HYB_EINVAL. */
    int32_t y0;             /* first global DSMC row of the slab (ncy_global > 0) */
} hyb_params;

/* Constants derived from hyb_params (hyb_derive). */
typedef struct {
    double r_lat;    /* c / c_s of the lattice: sqrt(3/2) (D3Q39) or sqrt(3) (D3Q19) */
    double cs_lat;   /* lattice sound speed in lattice units, 1 / r_lat */
    double H_lat;    /* LB nodes across the channel */
    double tau;      /* relaxation time, Eq. tau: sqrt(pi/8) (c/c_s) Kn H + 1/2 */
    double dt;       /* step in cell / c_th units: cs_lat / lb_ratio */
    double lambda;   /* mean free path in DSMC cells: Kn * ncx */
    double coll_dt;  /* F_N sigma_T dt / V_c of Eq. collisionnumber: dt / (sqrt(2) lambda ppc) */
    double g_step;   /* body-force velocity increment per step, 8 (tau-1/2) Ma cs^2 / H^2 */
    double c_th_ms;  /* sqrt(k T / m) [m/s] */
    int64_t ncells, nx, ny, nnodes;
    int64_t capacity; /* particle slots: ncells * bin */
    int32_t q, order;
    int32_t bin;      /* particle slots per cell */
    int32_t pad;
    int64_t nz;       /* LB layers along z: 1 for the slab, ncz * lb_ratio in 3D */
    int64_t ncz;      /* DSMC cells along z: 1 for the slab */
    int64_t yh;       /* LB ghost rows below and above the rows of a streamwise slab context (the
                         lattice's largest speed: 3 for D3Q39, 1 for D3Q19); 0 otherwise. The
                         lattice then has ny = ncy lb_ratio + 2 yh rows and node row y holds the
                         slab's LB row y - yh */
    int64_t xcap;     /* particles each exchange buffer of a slab holds (0 otherwise) */
} hyb_derived;

/* Byte offsets of the arrays inside the caller's arena (hyb_layout_compute). Arrays marked
 * [2] are ping-pong pairs; hyb_current says which half holds the current state. Real is
 * float or double per real_bytes. Particles are binned by cell: cell c owns slots
 * [c * bin, (c + 1) * bin) of every particle array and count[half][c] of them are in use,
 * in the order of their order keys (after dsmc_step; see part) or of their generation (after
 * dsmc_init and map_lbm_to_dsmc); the other half's counts are zero between calls.
 *   part          Real[ncells*bin][8]  particle records: x, y (positions in cell units, x
 *                                   across, y streamwise), vx, vy, vz (velocities in c_th
 *                                   units), z (3D only; else 0), the bits of a u32 order key
 *                                   (written by the move, scratch within a step: o * bin + rank
 *                                   for a particle displaced by at most one cell along every
 *                                   axis, o = (3 (dz+1) + dy+1) 3 + dx+1 its neighbour offset;
 *                                   else 2^31 + origin slot c * bin + rank; the collide orders
 *                                   a cell's arrivals by it) and one unused value; [2]
 *   count         u32[ncells]       particles per cell; [2]
 *   crmax         Real[ncells]      (sigma_T c_r)_max / sigma_T per cell
 *   rem           Real[ncells]      NTC fractional candidate carried between steps
 *   nbar_sum      u32[ncells]       running sum of N per cell, for N-bar
 *   acc           f64[ncells][20]   cumulative sums N, S v (3), S vv (6: xx xy xz yy yz zz),
 *                                   S vvv (10: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)
 *   f             Real[q][nz][ny][nx]  populations, x fastest (nz = 1 for the slab); [2]
 *   ctrl          u32[16]           [0] status bits, [1] particles in use, [2] DSMC steps
 *                                   taken, [3] moment samples taken, [4]..[15] scratch
 *   counters      u64[16]           event counters, HYB_C_*
 *   map_scratch                     LB2DSMC per-cell Grad records (FP64: rho, new count,
 *                                   a2[6], a3[10], u[3], C; 176 bytes per listed cell)
 *   coupled       u8[ncells]        coupling cells of a multi-step hybrid call in progress
 *                                   (zero between calls)
 */
typedef struct {
    uint64_t total_bytes;
    int64_t capacity, ncells, nnodes;
    int32_t q, real_bytes, bin, pad;
    uint64_t part[2], count[2];
    uint64_t crmax, rem, nbar_sum, acc;
    uint64_t f[2];
    uint64_t ctrl, counters, map_scratch;
    uint64_t coupled;
    uint64_t coll_cell;     /* Real[ncells]: per-cell NTC factor (kn_profile = 1; size 0 otherwise) */
    uint64_t tau_node;      /* Real[nnodes]: per-node relaxation time (kn_profile = 1) */
    /* exchange buffers of a streamwise slab (size 0 otherwise), xbytes each: a u32 count, then
     * xcap particle records (Real[8], as part) from byte 256, then xcap u32 channel cell ids
     * (the particle's new cell) */
    uint64_t xsend[2], xrecv[2], xbytes;
} hyb_layout;

typedef struct hyb_ctx hyb_ctx; /* opaque, owned by the library */

/* Host-only helpers (no GPU needed). Return HYB_EINVAL for invalid parameters (among the
 * limits: the channel's cells (ncx * rows * max(ncz, 1)) times 256 below 2^31, so that an
 * origin slot fits an order key's 31 bits). */
hyb_status hyb_derive(const hyb_params* p, hyb_derived* out);
hyb_status hyb_layout_compute(const hyb_params* p, hyb_layout* out);
/* The library's lattice: e[q][3] integer speeds, w[q] weights, r = c/c_s. Row order is the
 * population layout. `q` is 39 or 19; e and w must hold q rows. */
hyb_status hyb_lattice(int32_t q, int32_t* e, double* w, double* r);
const char* hyb_status_string(hyb_status s);

/* Create a context on the current CUDA device and initialise the state in `arena`:
 * ppc particles per cell, uniform inside the cell, Maxwellian at T (Sec. 3.1 "100
 * computational molecules are initially placed in each cell"), and the LB populations at
 * rest with density 1. `arena` is device memory of at least hyb_layout.total_bytes,
 * 256-byte aligned, owned by the caller. `stream` is a cudaStream_t (NULL: legacy default
 * stream; graph replay needs a non-default stream). On success *out owns the context. */
hyb_status dsmc_init(const hyb_params* p, void* arena, uint64_t arena_bytes, void* stream,
                     hyb_ctx** out);

/* `nsteps` DSMC steps (Sec. 5; the NTC order move -> index -> collide -> sample): each
 * particle is moved and binned into its new cell of the other half with its order key (see
 * part: the neighbour offset of its displacement, then its rank in its old cell), then every
 * cell puts its particles in the order of their keys, collides them and adds their moment
 * sums. With nsteps >= 2 the collide of each step and the move of the next may run as one
 * pass over the particles (hyb_set_fuse; the same results). Draws are keyed by (seed; cell,
 * step, purpose, index), so results do not depend on the launch shape. */
hyb_status dsmc_step(hyb_ctx* ctx, int32_t nsteps);

/* The passes of one DSMC step, for a streamwise slab (hyb_params.ncy_global > 0; the multi-GPU
 * decomposition of the channel into streamwise slabs) or any context. In this order:
 *   dsmc_move     moves and bins the particles (as dsmc_step); a slab's particles whose new
 *                 cell lies outside its rows go to its send buffers (xsend[0]: lower rows,
 *                 xsend[1]: higher rows, across the periodic end included) with their
 *                 order keys and channel cells;
 *                 -- the caller then copies each neighbour's send buffer into this slab's
 *                    receive buffer (xrecv[0] <- the slab below's xsend[1], xrecv[1] <- the
 *                    slab above's xsend[0]; hyb_layout.xbytes each, on this context's stream or
 *                    ordered before dsmc_merge), e.g. by NCCL send/recv between ranks --
 *   dsmc_merge    appends the received particles to their cells (a no-op for a context that
 *                 holds the whole channel) and clears the slab's send counts;
 *   dsmc_collide  orders, collides and samples every cell (as dsmc_step) and flips the
 *                 particle half.
 * dsmc_move + dsmc_merge + dsmc_collide of every slab give the whole channel's dsmc_step(1) bit
 * for bit. A call out of this order returns HYB_ESTATE; a received particle whose cell is not
 * the slab's raises HYB_ST_BAD_INPUT, a full send buffer or bin HYB_ST_CAPACITY. */
hyb_status dsmc_move(hyb_ctx* ctx);
hyb_status dsmc_merge(hyb_ctx* ctx);
hyb_status dsmc_collide(hyb_ctx* ctx);

/* LB ghost rows of a streamwise slab (the lattice's yh rows below and above the slab's rows,
 * hyb_derived.yh). Before each lbm_step of the slabs (and after any map_dsmc_to_lbm), every
 * slab packs, for each side (0: its lower boundary, 1: its upper one), the populations that
 * the neighbour on that side pulls across it (e_y < 0 at the lower boundary, e_y > 0 at the
 * upper one, from the |e_y| rows next to the boundary: only the outgoing populations), and
 * unpacks the neighbour's packed side into its own ghost rows (side 0: the buffer packed by the
 * slab below at its side 1; side 1: by the slab above at its side 0). lbm_halo_size gives the
 * values (Real) of one side's buffer: nz nx times the sum of the positive e_y (18 rows for
 * D3Q39, 5 for D3Q19). dev_buf is caller-owned device memory. HYB_EINVAL for a context that
 * holds the whole channel. */
hyb_status lbm_halo_size(const hyb_ctx* ctx, int64_t* values);
hyb_status lbm_halo_pack(hyb_ctx* ctx, int32_t side, void* dev_buf);
hyb_status lbm_halo_unpack(hyb_ctx* ctx, int32_t side, const void* dev_buf);

/* `nsteps` LB stream-collide steps (Sec. 2, Sec. 3.1). */
hyb_status lbm_step(hyb_ctx* ctx, int32_t nsteps);

/* Copy the cumulative moment sums acc[ncells][20] into `out` (device memory, may be NULL)
 * and, if `reset`, zero the sums and the sample count. The sums are ordered as in acc. */
hyb_status sample_moments(hyb_ctx* ctx, double* out, int32_t reset);

/* DSMC2LB (Sec. 2.1): for each LB node in dev_nodes[n] (device int32, node = y * nx + x,
 * distinct), overwrite its populations with the projection of the cumulative moments of the
 * DSMC cell that contains it: f_a = w_a sum_{n<=N} a^(n) : H^(n)(xi_a) / n! (Eq.
 * discretefunctions), a^(n) the raw Hermite coefficients of the sampled moments (FP64). */
hyb_status map_dsmc_to_lbm(hyb_ctx* ctx, const int32_t* dev_nodes, int32_t n);

/* LB2DSMC (Sec. 2.2, Table 1): for each DSMC cell in dev_cells[n] (device int32,
 * cell = iy * ncx + ix, distinct), replace its particles by floor(rho ppc + U) new ones,
 * with rho the mean LB density of the cell's lb_ratio^2 nodes; velocities drawn from the
 * Grad distribution of the cell's populations by acceptance-rejection with envelope
 * C = 1 + 30 M; positions uniform in the cell. The mean populations, rho, u and the Grad
 * coefficients are formed in FP64; the trials are evaluated in the state precision with the
 * coefficients rounded to it. A cell whose new count exceeds its bin keeps its particles and raises
 * HYB_ST_CAPACITY; an invalid cell index is skipped and raises HYB_ST_BAD_INPUT. */
hyb_status map_lbm_to_dsmc(hyb_ctx* ctx, const int32_t* dev_cells, int32_t n);

/* map_lbm_to_dsmc without any device memory of its own beyond the context's arena.
 * The paper has no counterpart: this entry point exists for callers that cannot give the
 * library more device memory or let it allocate, for example a host application whose own
 * allocator owns every byte of the GPU under a fixed budget, or a real-time loop that may not
 * call an allocator at all. It computes exactly what map_lbm_to_dsmc computes; its per-cell
 * Grad records go to a fixed array of HYB_NOALLOC_MAX_CELLS records (176 bytes each, about
 * 720 KB) compiled into the library, which every GPU that loads the library keeps until the
 * process exits. It calls no cudaMalloc, cudaFree or other allocating routine.
 * n > HYB_NOALLOC_MAX_CELLS returns HYB_EINVAL and launches nothing. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture, and call with the context's
 * device current (otherwise HYB_EINVAL). Calls outside a capture look the address up again,
 * so a call after cudaDeviceReset or from another context of the device uses its own
 * context's array; concurrent first calls from several host threads are serialised. Every call on a device shares the one array and it
 * keeps the last call's records: calls that overlap on the GPU (other streams or contexts on
 * the same device) race on it and must be serialised by the caller. */
#define HYB_NOALLOC_MAX_CELLS 4096
hyb_status map_lbm_to_dsmc_noalloc(hyb_ctx* ctx, const int32_t* dev_cells, int32_t n);

/* ---- Differentiated LBM (an extension beyond the paper) --------------------------------
 * The LB stream-collide of Sec. 2 (regularised BGK, kinetic walls, body force; tau from
 * Eq. tau) with a force increment g_y and a relaxation time tau per node, its adjoint, and a
 * coupling-interface loss: at each listed node, the 20 Grad coefficients of its populations
 * (rho; u = sum f xi / rho; a2 = sum f c c / rho - I and a3 = sum f c c c / rho with
 * c = xi - u, the comoving coefficients of Table 1; packed xx xy xz yy yz zz and xxx xxy xxz
 * xyy xyz xzz yyy yyz yzz zzz) against 20 targets, summed as squares. Populations and their
 * adjoints use the layout of the context's populations: [q][y][x], q < Q, nx * ny nodes,
 * state precision (real_bytes). g, tau and their gradients are one value per node in the
 * state precision. All buffers are device memory owned by the caller; every call is
 * enqueued on the context's stream; invalid pointers or sizes return HYB_EINVAL without
 * launching; the context's own populations are not touched. In 3D the populations are
 * [q][nz][ny][nx] and nodes (z ny + y) nx + x. */

/* One LB step f_dst = LB(f_src) with per-node g (force increment per step along the
 * streamwise axis) and tau. f_src and f_dst must differ. */
hyb_status lbm_step_nodes(hyb_ctx* ctx, const void* f_src, void* f_dst, const void* g_node,
                          const void* tau_node);

/* Interface loss of the populations f at the n listed nodes (node index y * nx + x) against
 * targets (n * 20 values): adds the loss to *dev_loss (one double, device) and adds dL/df
 * at the listed nodes to lam (populations-shaped; other entries untouched). A node index out
 * of range is skipped and raises HYB_ST_BAD_INPUT in the sticky status. */
hyb_status lbm_interface_loss(hyb_ctx* ctx, const void* f, const int32_t* dev_nodes, int32_t n,
                              const void* dev_targets, double* dev_loss, void* lam);

/* One step of the adjoint: with f the populations at step t and lam_next = dL/df_{t+1},
 * writes lam = dL/df_t (every entry) and adds dL/dg and dL/dtau of this step to grad_g and
 * grad_tau. wall is a scratch of 2 * ny * nz + 1 values (state precision; nz = 1 for the
 * slab) that must be zero before the first call; it is left zero. lam and lam_next must differ. The adjoint is that of the regularised
 * collision: a context with lb_collision = 1 returns HYB_EINVAL. */
hyb_status lbm_adjoint_step(hyb_ctx* ctx, const void* f, const void* lam_next, void* lam,
                            const void* g_node, const void* tau_node, void* grad_g,
                            void* grad_tau, void* wall);

/* nsteps LB steps in one call, as nsteps calls of lbm_step_nodes alternating between f_a
 * (holding f_0 on entry) and f_b: f_T ends in f_a when nsteps is even, else in f_b. The
 * states f_K, f_2K, ... before f_T (K = ckpt_every >= 1) are also copied to ckpt, one
 * population array each in order (floor((nsteps - 1) / K) of them; ckpt may be NULL when
 * there are none). HYB_EINVAL for nsteps < 0, ckpt_every < 1, f_a == f_b or a missing
 * pointer. */
hyb_status lbm_steps_nodes(hyb_ctx* ctx, void* f_a, void* f_b, const void* g_node, const void* tau_node,
                           int32_t nsteps, int32_t ckpt_every, void* ckpt);

/* The adjoint of n >= 1 LB steps from the state f_t0 (`state0`) in one call: the states
 * f_t0+1 .. f_t0+n-1 are recomputed into `states` (n - 1 population arrays of caller scratch;
 * NULL when n = 1), then n adjoint steps run from the last to the first, as n calls of
 * lbm_adjoint_step alternating between lam_a (dL/df_t0+n on entry) and lam_b: dL/df_t0 ends
 * in lam_a when n is even, else in lam_b. grad_g, grad_tau and wall as lbm_adjoint_step.
 * HYB_EINVAL for n < 1, lam_a == lam_b, a missing pointer or lb_collision = 1. */
hyb_status lbm_adjoint_segment(hyb_ctx* ctx, const void* state0, void* states, int32_t n, void* lam_a,
                               void* lam_b, const void* g_node, const void* tau_node, void* grad_g,
                               void* grad_tau, void* wall);

/* One or more hybrid steps: dsmc_step(1), map_dsmc_to_lbm, lbm_step(1), map_lbm_to_dsmc.
 * n_nodes or n_cells may be 0 to skip a mapping. With nsteps >= 2 the DSMC passes are fused
 * across steps: the collide of a step and the move of the next are one pass over the
 * particles, and LB2DSMC moves the particles it creates on at once; the results equal nsteps
 * single hybrid steps bit for bit (the state is complete only when the call's work is done).
 * With use_graph != 0 the work is replayed from a CUDA graph captured on first use (one step
 * per ping-pong parity, or, for nsteps >= 2 without kernel timing, the whole call per step
 * count and starting parities; recaptured if the arguments change); the stream must not be
 * the legacy default stream. */
hyb_status hyb_hybrid_step(hyb_ctx* ctx, const int32_t* dev_nodes, int32_t n_nodes,
                           const int32_t* dev_cells, int32_t n_cells, int32_t nsteps,
                           int32_t use_graph);

/* Adjoint of map_dsmc_to_lbm (Sec. 2.1, Eq. coefficients and Eq. discretefunctions, raw
 * coefficients; an extension beyond the paper, for the differentiated coupling). lam is
 * dL/df for the context's population layout ([q][nz][ny][nx], state precision, device),
 * taken right after map_dsmc_to_lbm wrote the n listed nodes (distinct, device int32).
 * Adds dL/d(acc) of the cells holding those nodes to grad_acc (device f64[ncells][20], the
 * layout of hyb_layout.acc) and sets lam at the listed nodes to zero, since the mapping
 * overwrote those populations. For a fixed sample count S (ctrl[3], which the forward call
 * used) the coefficients are linear in the sums, so acc itself is not read. A node index out
 * of range, or S = 0, is skipped and raises HYB_ST_BAD_INPUT. A context with d2l_mode = 1
 * (the equilibrium mapping) returns HYB_EINVAL. Enqueued on the context's stream. */
hyb_status map_dsmc_to_lbm_adjoint(hyb_ctx* ctx, const int32_t* dev_nodes, int32_t n, void* lam,
                                   double* grad_acc);

/* One hybrid step with the coupling lists and the results in HOST memory, for a host
 * application that holds its lists and reads the coupling moments every step. Enqueued on
 * the context's stream, in order:
 *   - the n_nodes nodes and n_cells cells (host int32) are copied to device staging owned by
 *     the context;
 *   - one hybrid step, as hyb_hybrid_step(ctx, staging, n_nodes, staging, n_cells, 1, 1);
 *   - the 20 cumulative moment sums of each listed cell (the layout of hyb_layout.acc; zeros
 *     for an index out of range) are copied to host_acc (n_cells x 20 doubles, list order);
 *   - the sticky status word (HYB_ST_* bits) is copied to *host_status.
 * The call returns once the work is enqueued; the host buffers must stay valid and
 * untouched until hyb_host_wait says the step is done. With page-locked host buffers
 * (cudaMallocHost, cudaHostRegister) the transfers are made by two kernels that read and
 * write the buffers through their device addresses, and the whole call is one CUDA graph
 * (as in hyb_hybrid_steps_host); host_acc and host_status must then be writable by the device
 * (not registered with cudaHostRegisterReadOnly). Pageable buffers work but take
 * cudaMemcpyAsync copies, which are then synchronous. The first call, and any call with longer lists, allocates
 * the staging (4 n_nodes + 164 n_cells bytes, rounded up) on the device; hyb_destroy frees
 * it. host_acc may be NULL when n_cells is 0. Invalid sizes or pointers: HYB_EINVAL. */
hyb_status hyb_hybrid_step_host(hyb_ctx* ctx, const int32_t* host_nodes, int32_t n_nodes,
                                const int32_t* host_cells, int32_t n_cells, double* host_acc,
                                uint32_t* host_status);

/* nsteps hybrid steps with host buffers in one call, as nsteps calls of hyb_hybrid_step_host
 * with the same lists (each step copies the lists in before its first kernel and its strip
 * sums and status out after its LB2DSMC), but with the DSMC passes of consecutive steps fused
 * as in hyb_hybrid_step (hyb_set_fuse, hyb_set_collide_block; the same results). host_acc
 * holds nsteps x n_cells x 20 doubles (step k's sums at k n_cells 20), host_status nsteps
 * words. With page-locked host buffers each step's transfers are two kernels (the lists read
 * from host memory, the sums and status written to it) and the call is enqueued as one CUDA
 * graph (captured at the first call with the same steps, lists, buffers and state halves; the
 * context keeps the two latest); pageable buffers take copies and direct launches. Either way
 * the call completes as one entry of the ring that hyb_host_wait counts. The staging and
 * errors are those of hyb_hybrid_step_host; nsteps < 1 is HYB_EINVAL. */
hyb_status hyb_hybrid_steps_host(hyb_ctx* ctx, int32_t nsteps, const int32_t* host_nodes, int32_t n_nodes,
                                 const int32_t* host_cells, int32_t n_cells, double* host_acc,
                                 uint32_t* host_status);

/* Waits until at most `pending` (0 to 3) of the steps issued by hyb_hybrid_step_host are
 * still in flight, so their results have landed in the host buffers: pending = 0 waits for
 * all of them, pending = 1 lets the newest run on while the host reads the one before. */
hyb_status hyb_host_wait(hyb_ctx* ctx, int32_t pending);

/* Which ping-pong halves hold the current particle and population state (0 or 1). */
hyb_status hyb_current(const hyb_ctx* ctx, int32_t* particle_half, int32_t* lb_half);

/* Whether dsmc_step and hyb_hybrid_step with nsteps > 1 fuse the collide of a step with the
 * move of the next (one pass over the particles per step). HYB_FUSE_AUTO (the default) fuses
 * when the fused pass's grid fills the GPU (at least as many blocks of 32 cells as are
 * resident at once), where it is faster; below that two passes per step are. The results are
 * the same bit for bit. HYB_EINVAL for another mode. */
#define HYB_FUSE_AUTO 0
#define HYB_FUSE_ALWAYS 1
#define HYB_FUSE_NEVER 2
hyb_status hyb_set_fuse(hyb_ctx* ctx, int32_t mode);

/* The collide's block shape: 8 warps for 32 cells (the default) or 4 warps for 16 (twice the
 * blocks per SM; the NTC chain of a block then runs on 16 lanes); HYB_EINVAL for others. The
 * shape changes no result. get returns the shape in use (-1 for a null context).
 * hyb_tune_collide times, for each shape, with and without fusion (HYB_FUSE_ALWAYS,
 * HYB_FUSE_NEVER), a captured eight-step hyb_hybrid_step with these lists (the best of four
 * replays, after the capture call and one replay), keeps the fastest pair and returns it in
 * *warps and *fuse (either may be NULL); it advances the context by 192 hybrid steps. */
hyb_status hyb_set_collide_block(hyb_ctx* ctx, int32_t warps);
int32_t hyb_get_collide_block(const hyb_ctx* ctx);
hyb_status hyb_tune_collide(hyb_ctx* ctx, const int32_t* dev_nodes, int32_t n_nodes,
                            const int32_t* dev_cells, int32_t n_cells, int32_t* warps, int32_t* fuse);

/* Synchronises. Returns the sticky device status mapped to a hyb_status (HYB_OK if clear),
 * and the raw bits in *bits if not NULL. */
hyb_status hyb_sync_status(hyb_ctx* ctx, uint32_t* bits);

/* Synchronises. Copies the HYB_NCOUNTERS event counters into out (host memory). */
hyb_status hyb_read_counters(hyb_ctx* ctx, uint64_t* out);

/* Kernel timing on the context's stream: after hyb_profile(ctx, k) every launch of kernel k
 * (0 move, 1 collide, 2 lbm, 3 dsmc2lb, 4 lb2dsmc, 5 the fused collide-and-move pass of
 * multi-step calls; -1 off) is bracketed by CUDA events. hyb_profile_harvest synchronises
 * and adds the elapsed times of the launches since the last harvest; call it after every
 * hybrid step when graphs are used. hyb_profile_read returns the totals. */
hyb_status hyb_profile(hyb_ctx* ctx, int32_t kernel);
hyb_status hyb_profile_harvest(hyb_ctx* ctx);
hyb_status hyb_profile_read(const hyb_ctx* ctx, double* total_ms, int64_t* launches);

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[4i..4i+3] = Philox(ctr[4i..4i+3],
 * key = (seed, seed >> 32)), for checking the generator against an independent one.
 * ctr and out are device pointers of n * 4 u32. */
hyb_status hyb_debug_philox(const uint32_t* dev_ctr, uint64_t seed, uint32_t* dev_out, int64_t n,
                            void* stream);

const char* hyb_last_error(const hyb_ctx* ctx);
/* Synchronises the stream, releases graphs and events; does not touch the arena. */
void hyb_destroy(hyb_ctx* ctx);

/* ---- Batched ensemble of independent channels ----------------------------------------
 * Beyond the paper's single channel (it names time or ensemble averaging as the remedy for
 * DSMC noise, Sec. 5): a batch advances n independent replicas, each with its own
 * hyb_params (sizes, ppc, Kn, seed...), with one launch per kernel for all of them per hybrid
 * step, replayed from a CUDA graph. The replicas share real_bytes and lattice. Replica r's
 * arena is the part of the caller-owned batch arena at offsets[r], with the layout of
 * hyb_layout_compute(&p[r]); a table region at offsets[n] holds the per-replica kernel
 * arguments and unit prefix sums, written by the library. A replica advanced in the batch
 * gives the same results as the same channel advanced alone. */
typedef struct hyb_batch hyb_batch;

/* offsets[0..n-1]: the replicas' arenas; offsets[n]: the table region; offsets[n+1]: the
 * total size. offsets has n + 2 entries. HYB_EINVAL for invalid parameters or replicas that
 * differ in real_bytes or lattice. */
hyb_status hyb_batch_layout(const hyb_params* p, int32_t n, uint64_t* offsets);

/* Initialises every replica (as dsmc_init) in the batch arena (256-byte aligned, at least
 * offsets[n+1] bytes) on `stream`. On success *out owns the batch. */
hyb_status hyb_batch_init(const hyb_params* p, int32_t n, void* arena, uint64_t arena_bytes,
                          void* stream, hyb_batch** out);

/* The context of replica r, owned by the batch (do not destroy it). Its views, counters and
 * status are those of the replica. A replica stepped on its own falls out of lockstep, and
 * the next batch step returns HYB_ESTATE. */
hyb_status hyb_batch_replica(hyb_batch* b, int32_t r, hyb_ctx** out);

/* nsteps hybrid steps of every replica (the order of hyb_hybrid_step). dev_nodes and
 * dev_cells are the replicas' coupling lists (device int32, each replica's own node and cell
 * indices) one after another; node_pre and cell_pre (host int64, n + 1 entries, starting at
 * 0) are their offsets. Empty lists skip a mapping for a replica. */
hyb_status hyb_batch_hybrid_step(hyb_batch* b, const int32_t* dev_nodes, const int64_t* node_pre,
                                 const int32_t* dev_cells, const int64_t* cell_pre,
                                 int32_t nsteps, int32_t use_graph);

/* Thread-block size of one kernel class of the batch, by the ids of hyb_profile (0 move: 64,
 * 128 or 256 threads; 1 collide: 256 for blocks of 32 cells or 128 for 16 cells, 8 lanes per
 * cell, as hyb_set_collide_block; 2 LB step: 32, 64 or 128; 3 DSMC2LB: 64, 128 or 256;
 * 4 LB2DSMC: 256, fixed by its design of 8 warps per cell); HYB_EINVAL for others. The results
 * do not depend on the shapes. get returns the size in use, -1 for an invalid id. */
hyb_status hyb_batch_set_block(hyb_batch* b, int32_t kernel, int32_t threads);
int32_t hyb_batch_get_block(const hyb_batch* b, int32_t kernel);

/* The move and LB block sizes in one call (hyb_batch_set_block for kernels 0 and 2). */
hyb_status hyb_batch_set_blocks(hyb_batch* b, int32_t move_block, int32_t lbm_block);

/* Autotuner: for each kernel class with more than one shape (move, collide, LB step,
 * DSMC2LB), one after another, times replayed hybrid steps of the batch at each of its block
 * sizes and keeps the fastest; returns the move and LB sizes (hyb_batch_get_block gives all).
 * The steps it times advance the batch (7 hybrid steps per shape tried, 77 in all). */
hyb_status hyb_batch_tune(hyb_batch* b, const int32_t* dev_nodes, const int64_t* node_pre,
                          const int32_t* dev_cells, const int64_t* cell_pre, int32_t* move_block,
                          int32_t* lbm_block);

const char* hyb_batch_last_error(const hyb_batch* b);
void hyb_batch_destroy(hyb_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* DSMCLBM_H */
