/*
 * lbm.h -- C ABI of the GB300 (sm_103a) reactive two-component lattice
 * Boltzmann library: capillary infiltration of a wetting melt with surface
 * reaction, precipitation and solid growth (Sergi, Grossi, Leidi, Ortona,
 * "Lattice Boltzmann simulation of the surface growth effects for the
 * infiltration of molten Si in carbon preforms", arXiv:1309.6726).
 *
 * One handle holds one lattice or a batch of independent lattices
 * ("capillaries") of uneven size; every call below acts on all of them.
 * The time step it runs is the paper's Sec. II model, per node and step:
 *
 *   streaming of the two D2Q9 populations and the D2Q4 solute with
 *   half-way bounce-back at the solid (the wall rule of Sec. II);
 *   densities and momenta;
 *   Martys-Chen cohesive (A-B) and adhesive (fluid-solid) forces,
 *     F_s = -G_c rho_s(x) sum_i w_i rho_s'(x+e_i) e_i
 *           - G_ads,s rho_s(x) sum_i w_i solid(x+e_i) e_i,
 *     G_ads,A = -g_ads, G_ads,B = +g_ads (the two interaction forces of
 *     Sec. II; g_ads sets the 30 degree contact angle of Sec. I);
 *   Shan-Chen velocity shift and BGK collision of each component;
 *   BGK collision of the D2Q4 solute advected by the barycentric velocity
 *     (the solute is carried by the flow without acting on it, Sec. II),
 *     with the inlet column
 *     x = 0 imposing concentration c_in when enabled;
 *   first-order surface reaction k_r at fluid nodes where A is the
 *     majority and that touch the solid: the consumed solute precipitates
 *     on the solid surface (Sec. II);
 *   growth: a node whose precipitated mass reaches m_threshold turns solid
 *     (the threshold rule of Sec. II); its fluid, solute and deposit go to
 *     a per-lattice ledger so that mass is accounted exactly.
 * Lattices are periodic in x and y; node (x, y) is row y, column x.
 *
 * Threading and streams: a handle is not thread-safe.  Calls that only
 * launch work (lbm_step) are asynchronous on the handle's stream (its own
 * non-blocking stream unless lbm_set_stream bound another); every call
 * that returns data to the host synchronizes that stream first.
 *
 * Errors: every call returns an lbm_status; on failure the handle keeps a
 * message that lbm_last_error returns.  Nothing throws across the ABI.  A
 * CUDA error leaves the handle unusable (LBM_ECUDA from then on).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,   /* bad argument (sizes, NULL, out-of-range index) */
    LBM_ENOMEM = 2,   /* device or host allocation failed */
    LBM_ECUDA = 3,    /* a CUDA call or kernel failed; handle is dead */
    LBM_ETIMEOUT = 4, /* a bounded device wait ran out */
    LBM_ENAN = 5,     /* non-finite density seen in some lattice */
    LBM_EIO = 6       /* checkpoint file could not be read or written */
} lbm_status;

/* Storage of the populations between steps.  Arithmetic is FP32 in both;
 * the deposit and the growth test are FP64 in both. */
typedef enum {
    LBM_FP32 = 0, /* populations stored as FP32 */
    LBM_FP16 = 1, /* populations stored as FP16 deviations from per-node
                     references exact in FP32: per component, direction i
                     reads back f_i / w_i = rho~ + e_i . v + 2^-10 d_i, with
                     rho~ = f_0 / w_0 (the rest population, FP32) and v
                     the odd part of the axis populations ((f^_1 -
                     f^_3) / 2, (f^_2 - f^_4) / 2, rounded to FP16) for
                     the component with the larger rest population where
                     |v_x| + |v_y| <= rho~, for the other one at nodes
                     next to a wall where |v_x| + |v_y| <= 4 rho~, else
                     0; so d_i holds only the second-order and
                     non-equilibrium part there;
                     the solute reads back 4 g_k = C~ + 2^-10 d_k.  The A and
                     B values of a direction share one 32-bit word; the
                     references take up the rounding of the deviations, so
                     each node keeps its mass to FP32 rounding.  15 32-bit
                     words per node against FP32's 22. */
    LBM_BF16 = 2  /* as LBM_FP16 with BF16 (8-bit significand, FP32's
                     exponent range) in place of FP16 for the deviations
                     and the linear term: the same layout and bytes, eight
                     times coarser rounding of the deviations. */
} lbm_precision;

/* Geometry and initial state of one lattice.  Arrays are row-major ny*nx,
 * read once at create (the caller keeps ownership).  Every fluid node
 * starts at rest equilibrium for its rho_a, rho_b and conc; values at solid
 * nodes are ignored.  [cap_x0, cap_x1) is the capillary section the
 * observables of Sec. III (front, radii, Delta e, closure) are taken over;
 * walls are expected at rows 0 and ny-1 there. */
typedef struct lbm_geometry {
    int32_t nx, ny;        /* nx >= 1, ny >= 3 */
    const uint8_t *solid;  /* 1 = solid, 0 = fluid */
    const float *rho_a;    /* initial density of component A (wetting) */
    const float *rho_b;    /* initial density of component B */
    const float *conc;     /* initial solute concentration */
    int32_t cap_x0, cap_x1;/* 0 <= cap_x0 < cap_x1 <= nx */
} lbm_geometry;

/* Model constants of one lattice (lattice units). */
typedef struct lbm_params {
    double tau_a, tau_b;  /* BGK relaxation times of A and B, > 1/2 */
    double tau_d;         /* solute relaxation time, D = (tau_d - 1/2)/2 */
    double g_coh;         /* cohesion strength G_c */
    double g_ads;         /* adhesion strength g (A attracted for g > 0) */
    double k_r;           /* reaction-rate constant [lu/ts], >= 0 */
    double m_threshold;   /* precipitated mass that turns a node solid, > 0 */
    double c_in;          /* concentration imposed at the inlet column */
    double body_force_x;  /* uniform acceleration along x (checks only) */
    int32_t inlet;        /* 1: column x = 0 imposes c_in */
    int32_t precision;    /* lbm_precision; must be equal over a batch */
} lbm_params;

/* Observables of one lattice at the current step (paper Sec. III).
 * front: centerline position of the A/B front past the capillary
 *   entrance (Fig. 2, Eq. 1), linear interpolation of rho_A - rho_B on the
 *   centerline row(s), NaN if there is none;
 * wetted_lower / wetted_upper: fluid nodes along each wall profile in the
 *   section where A is the majority;
 * r_min, r_ave: minimum and mean half-aperture; r_h: fluid area between
 *   the lower-wall profile and the centerline over that profile's length
 *   (Fig. 4); delta_e: largest grown wall thickness, H/2 for a closed
 *   column (Fig. 3);
 * precip_mass: all mass precipitated so far; mass_a/b/c: A, B and solute
 *   in the fluid; ledger_*: what growth moved out of the fluid;
 * closed: some section column is entirely solid; closure_step: the first
 *   step count at which that happened (-1 if never); nonfinite: a
 *   non-finite density was seen. */
typedef struct lbm_obs {
    int64_t step;
    double front;
    double wetted_lower, wetted_upper;
    double r_min, r_h, r_ave;
    double delta_e;
    double precip_mass;
    double mass_a, mass_b, mass_c;
    double ledger_a, ledger_b, ledger_c, ledger_m;
    int32_t closed;
    int32_t nonfinite;
    int64_t closure_step;
} lbm_obs;

/* Field selectors for lbm_get_fields / lbm_set_fields.  Populations are
 * the post-streaming state at the current step, FP32, direction-major:
 *   LBM_FIELD_POPS: 22 planes of ny*nx floats: A (9, D2Q9 order below),
 *                   B (9), solute (4);
 *   LBM_FIELD_DEPOSIT: ny*nx doubles;
 *   LBM_FIELD_DENSITY: 3 planes of ny*nx floats: rho_A, rho_B, C.
 * D2Q9 order: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1);
 * D2Q4 order: (1,0) (0,1) (-1,0) (0,-1).  Solid nodes read as zero. */
enum {
    LBM_FIELD_POPS = 0,
    LBM_FIELD_DEPOSIT = 1,
    LBM_FIELD_DENSITY = 2
};

typedef struct lbm_handle lbm_handle;

/* Creates a handle holding one lattice: the capillary or pore geometry and
 * the model constants of paper Sec. II (both fluids start at rest,
 * reading c13; the solute at the given concentration).  Copies the
 * geometry to the device (host->device once) and allocates everything the
 * steps need; *out is NULL on failure.  Returns EINVAL for bad sizes or
 * parameters, ENOMEM, ECUDA. */
lbm_status lbm_create(const lbm_geometry *g, const lbm_params *p,
                      lbm_handle **out);

/* Same for `count` independent lattices (g[k], p[k]) advanced together by
 * one launch per step over a packed ragged layout. */
lbm_status lbm_create_batch(const lbm_geometry *g, const lbm_params *p,
                            int32_t count, lbm_handle **out);

/* Binds a CUDA stream (a cudaStream_t passed as void*; NULL = the handle's
 * own stream).  The caller keeps the stream alive while bound. */
lbm_status lbm_set_stream(lbm_handle *h, void *cuda_stream);

/* Advances every lattice by n >= 0 time steps of the paper's Sec. II
 * update (collision with the Martys-Chen forces, streaming with half-way
 * bounce-back, solute advection-diffusion, surface reaction, deposit and
 * growth; readings c1-c12).  Asynchronous on the bound stream.  The last
 * step of a call (n > 0) also adds up each lattice's fluid content (rho_A,
 * rho_B and C over the nodes it updates), which the next lbm_observables
 * then reads instead of every node's populations. */
lbm_status lbm_step(lbm_handle *h, int64_t n);

/* Number of completed steps. */
int64_t lbm_step_count(const lbm_handle *h);

/* Number of lattices in the handle. */
int32_t lbm_count(const lbm_handle *h);

/* Observables of every lattice: out[count].  Synchronizes.  Returns
 * LBM_ENAN (after filling out) if some lattice holds a non-finite value.
 * The fluid content (mass_a, mass_b, mass_c) comes from the totals of the
 * last lbm_step call when no call has changed the state since (after
 * lbm_create, lbm_load, lbm_set_fields or lbm_autotune it sums the stored
 * populations instead); the two agree to FP32 rounding of each node's
 * sums. */
lbm_status lbm_observables(lbm_handle *h, lbm_obs *out);

/* Current solid mask of lattice k (the grown solid of paper Sec. II-III,
 * 1 = solid): n must be ny*nx bytes, row-major.  Synchronizes. */
lbm_status lbm_get_solid_mask(lbm_handle *h, int32_t k, uint8_t *host,
                              size_t n);

/* Current solid masks of every lattice of the handle, one call: each
 * lattice's ny*nx bytes (row-major, 1 = solid) back to back in lattice
 * order; n must be the sum of nx*ny.  Project addition (one device pass
 * and one copy for a whole batch).  Synchronizes. */
lbm_status lbm_get_solid_masks(lbm_handle *h, uint8_t *host, size_t n);

/* Copies a field of lattice k (see LBM_FIELD_*; the post-streaming
 * populations the Sec. II update is stated in, the deposit, the densities)
 * to host memory of exactly `bytes` bytes.  Project addition for parity
 * checks and analysis.  Synchronizes. */
lbm_status lbm_get_fields(lbm_handle *h, int32_t k, int32_t which,
                          void *host, size_t bytes);

/* Replaces the post-streaming populations (LBM_FIELD_POPS) or the deposit
 * (LBM_FIELD_DEPOSIT) of lattice k.  Values at solid nodes are ignored; a
 * deposit outside [0, m_threshold) at a fluid node is LBM_EINVAL (such a
 * node would already have turned solid). */
lbm_status lbm_set_fields(lbm_handle *h, int32_t k, int32_t which,
                          const void *host, size_t bytes);

/* Checkpoint and resume (project addition; the paper has no counterpart).
 * Writes / reads the complete device state (populations in their stored
 * precision, mask, deposit, ledgers, counters, step) to / from a file; a
 * loaded handle continues bit for bit as the saved one would have.  The
 * handle given to lbm_load must have been created with the same
 * geometry sizes and parameters. */
lbm_status lbm_save(lbm_handle *h, const char *path);
lbm_status lbm_load(lbm_handle *h, const char *path);

/* Step-kernel variant in use: kernel 0 = direct global loads, 1 =
 * TMA-staged tiles (default); tile of tx by ty nodes per block. */
typedef struct lbm_tuning {
    int32_t kernel;
    int32_t tx, ty;
    double ms_per_step;  /* measured by lbm_autotune, 0 otherwise */
} lbm_tuning;

/* Autotuner for the step kernel (project addition; the paper describes no
 * implementation).  Times every supported variant (direct or TMA-staged,
 * tile shapes 32x4, 32x8, 32x16, 64x4, 64x8, 128x4) for `steps` steps on this
 * handle's own state, restores the state after each trial, and keeps the
 * fastest; every variant computes bit-identical results, so only speed
 * differs.  Synchronizes; allocates a temporary copy of the state for the
 * trials.  out (may be NULL) receives the choice.  steps >= 1. */
lbm_status lbm_autotune(lbm_handle *h, int32_t steps, lbm_tuning *out);

/* The variant in use. */
lbm_status lbm_get_tuning(const lbm_handle *h, lbm_tuning *out);

/* Frees everything; NULL is allowed. */
void lbm_destroy(lbm_handle *h);

/* Message of the last failure on h (or of the last failed create when h is
 * NULL); never NULL. */
const char *lbm_last_error(const lbm_handle *h);

/* Effective radius (paper Sec. III, Fig. 4): Eq. 1's late-time speed
 * v = gamma H cos(theta) / (6 mu L) solved for H with v the least-squares
 * slope of the front history z(t) (n >= 2 samples), r_eff = H / 2.
 * Host-only arithmetic. */
lbm_status lbm_fit_reff(const double *t, const double *z, int32_t n,
                        double gamma, double mu, double length,
                        double cos_theta0, double *r_eff);

/* Tile schedule of the TMA-staged step kernel (project addition; the paper
 * describes no implementation), computed on the host as lbm_create computes
 * it: the tiles of tx by ty nodes of `count` lattices of nx[l] by ny[l]
 * nodes, dealt to `grid` persistent blocks.  A strip is a run of tiles down
 * one tile column of a lattice; columns longer than
 * max(4, ceil(tiles / (4 grid))) tiles are cut into strips of that length,
 * and strips go, longest first, to the block with the fewest tiles so far
 * (ties to the lower index).  Block b's k-th tile is written to
 * out[3 * (k * grid + b) + 0, 1, 2] = lattice, first column, first row;
 * lattice -1 (columns and rows 0) follows a block's last tile.  *slots
 * receives the longest list, so out holds 3 * grid * *slots values; out may
 * be NULL to query *slots alone, else it holds cap int32 values
 * (LBM_EINVAL when fewer than needed).  LBM_EINVAL for NULL nx, ny or
 * slots, count, tx, ty or grid < 1, or a lattice size < 1.  Host-only
 * arithmetic: needs no GPU. */
lbm_status lbm_plan_tiles(const int32_t *nx, const int32_t *ny, int32_t count,
                          int32_t tx, int32_t ty, int32_t grid, int32_t *out,
                          int64_t cap, int32_t *slots);

/* ---- observables without allocation ----------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code running inside a memory pool or
 * arena that another runtime owns (a framework's caching allocator), builds
 * that forbid dynamic allocation after start-up, or code that must not
 * synchronize the device, as cudaMalloc and cudaFree may.  Such callers
 * cannot create a handle (lbm_create allocates), so this call takes one
 * lattice's state as device pointers and writes the observables to a
 * device pointer.  It computes what lbm_observables reports for a handle in
 * the same state.
 *
 * pops:    [22][ny][nx] FP32 post-streaming populations (LBM_FIELD_POPS
 *          layout), device memory;
 * solid:   [ny][nx] current solid mask (1 = solid), device memory;
 * solid0:  [ny][nx] initial solid mask (wall thickness reference);
 * deposit: [ny][nx] precipitated mass (doubles), device memory;
 * ledger:  host array of 4 doubles, mass moved out of the fluid by growth
 *          (A, B, solute, deposit); copied into the result;
 * step, closure_step: copied into the result;
 * out:     one lbm_obs in device memory, written by the call;
 * cuda_stream: the stream the two kernels are launched on (NULL = the
 *          legacy default stream); the call is asynchronous on it.
 *
 * Allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).  Its working memory is a file-scope device array of
 * LBM_STATIC_MAX_COLUMNS column records (about 1.44 MB) that every GPU
 * which loads this library holds until the process exits; nx above that
 * limit returns LBM_EINVAL.  The first call on a device looks up the
 * array's device address, with that device current; make that first call
 * before any stream capture.  All calls on a device share the array:
 * calls whose kernels overlap on the GPU (different streams, or different
 * host threads) race and must be serialized by the caller.  Each call
 * writes every record it reads, so no clearing is needed between calls.
 * The result's nonfinite flag covers only the state passed in (a handle's
 * lbm_observables also keeps a flag set by earlier steps, e.g. at a node
 * that has since turned solid).
 * Returns LBM_EINVAL for NULL pointers or bad sizes, LBM_ECUDA if the
 * set-up or the launch fails, or if a CUDA error was already pending when
 * the call was made (nothing is launched then and the pending error is not
 * cleared). */
#define LBM_STATIC_MAX_COLUMNS 16384
lbm_status lbm_observables_static(const float *pops, const uint8_t *solid,
                                  const uint8_t *solid0,
                                  const double *deposit, int32_t nx,
                                  int32_t ny, int32_t cap_x0, int32_t cap_x1,
                                  const double ledger[4], int64_t step,
                                  int64_t closure_step, lbm_obs *out,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
