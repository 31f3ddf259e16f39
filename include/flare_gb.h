/*
 * flare_gb.h -- C ABI of the GB300 (sm_103a) implementation of the FLARE
 * mapped sparse-GP force field's per-step hot path: cell-list neighbour
 * search, normalized ACE-B2 descriptors, mapped energy and variance, and
 * forces by the reordered chain rule.
 *
 * Paper: "Micron-scale heterogeneous catalysis with Bayesian force fields
 * from first principles and active learning" (arXiv 2204.12573), Sec. V-B
 * (descriptors, kernel, mapped sparse GP, Eq. 1 and Eq. 2, force reordering,
 * multi-element compaction) and Sec. V-C (atom batching, neighbour lists).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an int status: FLR_OK (0) or one of the FLR_E*
 *   codes below.  On error, flr_last_error() returns a message for the
 *   calling thread; the message stays valid until the next call on that
 *   thread.
 * - All per-atom arrays are DEVICE pointers owned by the caller (for example
 *   torch tensors), except the HOST arrays of flr_host_state and of the
 *   server's requests.  The library never frees them and never keeps them
 *   past the call, except where stated for flr_md_state and flr_host_state
 *   (asynchronous copies).
 * - Calls that take a cudaStream_t enqueue work on that stream and return
 *   without synchronizing, unless stated otherwise.  Errors found on the
 *   device (neighbour-list overflow, non-finite forces, internal wait
 *   timeouts) are recorded in a device status word and reported by the
 *   next flr_sync() on the context.
 * - Units: Angstrom, eV, amu, ps.  Species are 0 .. n_species-1
 *   (0 = Pt, 1 = H in the H2/Pt(111) workload).
 * - Descriptor component order (full layout, dimension d_full):
 *   index = tri(a, b) * (l_max + 1) + l for radial channels
 *   a = s * n_max + n, a <= b, tri() row-major over the upper triangle.
 */
#ifndef FLARE_GB_H
#define FLARE_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *flr_stream_t; /* == cudaStream_t; NULL = legacy default stream */

/* status codes */
#define FLR_OK 0
#define FLR_EINVAL 1           /* invalid argument or unsupported parameter */
#define FLR_ENOMEM 2           /* device allocation failed */
#define FLR_ECUDA 3            /* CUDA runtime error (message has the CUDA error string) */
#define FLR_ENBR_OVERFLOW 4    /* an atom has more neighbours than max_nbr; rebuild with a larger max_nbr */
#define FLR_ETIMEOUT 5         /* a device-side wait gave up (kernel returned early; results invalid) */
#define FLR_EBUDGET 6          /* request exceeds the configured memory budget */
#define FLR_EDEVICE 7          /* device-detected invalid data (non-finite force, image shift out of range) */
#define FLR_ENOMODEL 8         /* flr_set_model() not called for every species */

/* quadratic-form precision (Eq. 1 and Eq. 2 evaluated as GEMMs) */
#define FLR_PREC_FP32 0        /* FP32 SIMT GEMM (the plain path) */
#define FLR_PREC_TF32 1        /* tcgen05 kind::tf32, FP32 accumulate in tensor memory */
#define FLR_PREC_BF16X3 2      /* tcgen05 kind::f16, hi/lo BF16 split, 3 products, FP32 accumulate */

/* How the variance quadratic form V = d^T Sigma d (Eq. 2) is evaluated.
 * DIRECT: the GEMM forms Sigma d and V = d . (Sigma d) in FP32.
 * AUTO (the default): as DIRECT, and every atom whose V may have lost its
 * digits gets V re-evaluated in FP64 from its FP32 descriptor and an FP64
 * copy of Sigma (FLR_TOT_N_VAR_FP64 counts them): V below 1/32 of
 * sum_k |d_k (Sigma d)_k| (the final sum cancelled), or V below 2e-3 (FP32
 * GEMM) or 2e-2 (3xBF16) of |Sigma_c|_2 (the GEMM's absolute error scales
 * with |Sigma_c|_2; this is how an ill-conditioned Sigma with d near its
 * small-eigenvalue directions shows).  TF32 applies the first test only.  flr_set_model checks that Sigma is
 * positive semi-definite (FP64 Cholesky).  FACTORED: the GEMM forms L^T d
 * with Sigma_c = L L^T the Cholesky factor of each compaction class's block
 * and V = |L^T d|^2, a sum of squares (no FP64 on the device). */
#define FLR_VAR_AUTO 0
#define FLR_VAR_DIRECT 1
#define FLR_VAR_FACTORED 2

/* indices into the per-evaluation totals array (double[FLR_NTOTALS], device) */
#define FLR_TOT_ENERGY 0       /* sum_i E_i (eV), FP64 */
#define FLR_TOT_VIRIAL 1       /* 9 entries, W_ab = -sum_pairs (r_ij)_a (dE_i/dr_ij)_b (eV), FP64 */
#define FLR_TOT_MAX_SIGMA 10   /* max_i sqrt(V_i) */
#define FLR_TOT_N_ISOLATED 11  /* atoms with no neighbour inside r_cut (descriptor defined as 0) */
#define FLR_TOT_KINETIC 12     /* sum_i m_i v_i^2 / 2 (eV), written by flr_md_step only */
#define FLR_TOT_N_REBUILDS 13  /* neighbour-list rebuilds performed by the last flr_md_step call */
#define FLR_TOT_N_VAR_FP64 14  /* atoms whose variance was re-evaluated in FP64 (FLR_VAR_AUTO) */
#define FLR_TOT_N_UNCERTAIN 15 /* flr_md_step: atoms with sigma > sigma_stop at the last step run */
#define FLR_TOT_N_CN 16        /* flr_md_step: atoms of species cn_species with a same-species
                                  neighbour closer than cn_cutoff (2 per intact H2 molecule) */
#define FLR_TOT_THERMOSTAT 17  /* flr_md_step (NVT): Q xi^2 / 2 + g kB T eta (eV); with the
                                  potential and kinetic energies this sum is conserved */
#define FLR_NTOTALS 24

typedef struct flr_ctx flr_ctx;
typedef struct flr_nbrlist flr_nbrlist;

/* Model hyperparameters (Sec. V-B).  Supported: n_species = 2, n_max in
 * {7, 8}, l_max = 3, max_nbr a multiple of 32 in [32, 512]. */
typedef struct {
    int32_t n_species;   /* chemical species S */
    int32_t n_max;       /* radial functions N (Chebyshev T_0 .. T_{N-1} of 2r/r_cut - 1) */
    int32_t l_max;       /* maximum angular momentum L of the real spherical harmonics */
    int32_t max_nbr;     /* neighbour-list row capacity per atom */
    double r_cut;        /* descriptor cutoff (A); cutoff function (r_cut - r)^2 */
    double skin;         /* Verlet skin (A); the list holds pairs closer than r_cut + skin */
    int32_t precision;   /* FLR_PREC_* */
    int32_t compaction;  /* 1: species-block compaction (Sec. V-B), 0: every atom uses d_full */
} flr_params;

/* One atomic structure.  pos: device float[n_atoms][4] (x, y, z, unused),
 * 16-byte aligned.  species: device int32[n_atoms].  cell: host, rows are
 * the lattice vectors a1, a2, a3.  pbc[d] != 0 makes direction d periodic;
 * along periodic directions positions should lie inside the cell (the
 * neighbour build accepts image offsets up to 2 cells). */
typedef struct {
    int32_t n_atoms;
    const float *pos;
    const int32_t *species;
    double cell[9];
    int32_t pbc[3];
} flr_system;

/* A batch of structures evaluated together (different sizes and cells):
 * atoms of structure s are rows offsets[s] .. offsets[s+1]-1 of pos and
 * species.  pos: device float[n_atoms][4], 16-byte aligned; species: device
 * int32[n_atoms]; offsets: host int32[n_structs + 1] with offsets[0] = 0 and
 * offsets[n_structs] = n_atoms; cells: host double[n_structs][9] (rows are
 * lattice vectors); pbc: host int32[n_structs][3]. */
typedef struct {
    int32_t n_structs;
    int32_t n_atoms;
    const float *pos;
    const int32_t *species;
    const int32_t *offsets;
    const double *cells;
    const int32_t *pbc;
} flr_batch;

/* Per-atom results (device pointers; any may be NULL except forces). */
typedef struct {
    float *energy;       /* [n] E_i = d^T beta_{s_i} d (Eq. 1, mapped) */
    float *forces;       /* [n][3] F_i = -dE/dr_i */
    float *variance;     /* [n] V_i = d^T Sigma_{s_i} d (Eq. 2, mapped) */
    float *sigma;        /* [n] sqrt(V_i): the predictive uncertainty */
    double *totals;      /* [FLR_NTOTALS] reductions, see FLR_TOT_* */
} flr_outputs;

/* MD state for flr_md_step (velocity Verlet).  pos and vel are device
 * float[n][4] updated in place; vel[.][3] is unused.  The forces buffer of
 * the flr_outputs passed to flr_md_step must hold the forces of the current
 * positions when forces_valid != 0; otherwise they are computed first. */
typedef struct {
    int32_t n_atoms;
    float *pos;
    float *vel;
    const int32_t *species;
    double cell[9];
    int32_t pbc[3];
    double masses[8];       /* amu, per species */
    double dt;              /* ps (0.0005 = 0.5 fs) */
    int32_t rebuild_every;  /* forced rebuild cadence in steps (plus max displacement > skin/2) */
    int32_t forces_valid;   /* set to 1 by flr_md_step on return */
    int64_t step;           /* running step counter, advanced by flr_md_step */
    /* Nose-Hoover thermostat (NVT; Sec. VI-A runs at fixed temperature):
     * temperature > 0 turns it on, tau is its period (ps); xi (1/ps) and eta
     * (its time integral) are the thermostat state, kept here between calls. */
    double temperature;
    double tau;
    double xi, eta;
    /* Uncertainty-triggered stop (the on-the-fly learning trigger of Sec. II):
     * sigma_stop > 0 ends the call after the first step at which some atom's
     * sigma exceeds it (halted = 1; FLR_TOT_N_UNCERTAIN counts the atoms). */
    double sigma_stop;
    int32_t halted;
    /* Coordination count for reaction monitoring: atoms of species
     * cn_species with a neighbour of the same species closer than cn_cutoff
     * (A) at the last step (FLR_TOT_N_CN); cn_species < 0 turns it off. */
    int32_t cn_species;
    double cn_cutoff;
} flr_md_state;

/* Thread-local text of the last error on the calling thread. */
const char *flr_last_error(void);

/* Library version string. */
const char *flr_version(void);

/* Create a context on CUDA device `device` (allocates the device status
 * word; model and workspace are allocated later).  *out is owned by the
 * caller and released with flr_destroy. */
int flr_create(const flr_params *params, int device, flr_ctx **out);

/* Release a context and every device buffer it owns (not the nbrlists). */
int flr_destroy(flr_ctx *ctx);

/* Descriptor dimensions: d_full = C(C+1)/2 (L+1) with C = S*N, and
 * d_single = N(N+1)/2 (L+1) for a one-species environment (Sec. V-B:
 * 420 and 112 for N = 7, L = 3). */
int flr_descriptor_dims(const flr_ctx *ctx, int32_t *d_full, int32_t *d_single);

/* Switch the quadratic-form precision of an existing context. */
int flr_set_precision(flr_ctx *ctx, int32_t precision);

/* Context options (flr_set_option).
 * FLR_OPT_FUSED_ONE_SPECIES: 1 evaluates the atoms of the
 * one-species compaction classes (Sec. V-B: most atoms of a slab) with one
 * kernel that computes their descriptors, writes them as the BF16 hi/lo
 * operand tile of the tensor cores in shared memory, and runs the quadratic
 * forms and their epilogue (E, V, sigma, dE/dB) from there, so their
 * descriptor rows never reach device memory; used with FLR_PREC_BF16X3 and
 * compaction on.  0 (default): descriptor and quadratic-form kernels run
 * separately.
 * Results agree within the 3xBF16 error (the epilogue uses the hi + lo
 * descriptor instead of the FP32 one). */
#define FLR_OPT_FUSED_ONE_SPECIES 1
/* FLR_OPT_OVERLAP_TWO_SPECIES: 1 (default) launches the one-species
 * quadratic-form kernel as a programmatic dependent of the two-species one
 * before it (Sec. V-B compaction classes; the two-species classes hold a few
 * atoms of a slab, at the full descriptor length), so it starts on the SMs
 * the two-species tiles leave free instead of after them; with
 * FLR_PREC_BF16X3 and compaction on.  Everything stays on the caller's
 * stream.  0: one kernel after the other.  Results are bitwise the same
 * either way. */
#define FLR_OPT_OVERLAP_TWO_SPECIES 2
int flr_set_option(flr_ctx *ctx, int32_t option, int32_t value);

/* Upload the mapped model of central species `species` (Eq. 1, Eq. 2):
 * beta and sigma are HOST double[d_full][d_full], row-major, symmetric
 * (the library uses (M + M^T)/2 and reports the largest asymmetry through
 * flr_last_error as information).  Builds the per-class compacted blocks
 * and the FP32 / BF16-hi/lo copies on the device.  Synchronous. */
int flr_set_model(flr_ctx *ctx, int32_t species, const double *beta, const double *sigma);

/* Map a sparse GP of central species `species` onto the quadratic forms and
 * install it (Sec. V-B, "Mapped Sparse GP"; Eq. 1 and Eq. 2 reordered):
 *   beta  = sig2 * D_S^T diag(alpha) D_S,
 *   Sigma = sig2 * I - sig2^2 * D_S^T K_SS^{-1} D_S,
 * so that d^T beta d equals the Eq. 1 sum over the sparse set
 * sig2 * sum_s alpha_s (d . d_s)^2 and d^T Sigma d the Eq. 2 variance
 * sig2 - sig2^2 k^T K_SS^{-1} k with k_s = d . d_s (unit d).  All in FP64 on
 * the device: Cholesky K_SS = L L^T, X = L^{-1} D_S, Sigma from X^T X.
 *   d_sparse: DEVICE double[n_sparse][d_full], the sparse set's normalized
 *             descriptor rows in the ABI component order (as returned by
 *             flr_compute_descriptors);
 *   alpha:    DEVICE double[n_sparse], the mean weights;
 *   k_ss:     DEVICE double[n_sparse][n_sparse], symmetric positive
 *             definite (only its lower triangle is read);
 *   sig2:     the signal variance sigma^2 > 0;
 *   beta_out, sigma_out: optional DEVICE double[d_full][d_full] copies of
 *             the mapped matrices (NULL to skip).
 * The inputs are not modified; temporary device memory of
 * 8 (n_sparse^2 + n_sparse d_full + 2 d_full^2) bytes is allocated and freed.
 * Then behaves as flr_set_model with the mapped matrices (its checks apply).
 * FLR_EINVAL if K_SS is not positive definite (a Cholesky pivot <= 0).
 * Synchronous on `stream`. */
int flr_map_sgp(flr_ctx *ctx, int32_t species, int32_t n_sparse, const double *d_sparse, const double *alpha,
                const double *k_ss, double sig2, double *beta_out, double *sigma_out, flr_stream_t stream);

/* Choose the variance evaluation (FLR_VAR_*) for models set afterwards and
 * re-upload the models already set.  FLR_EINVAL if a Sigma block is not
 * positive semi-definite (its Cholesky factorization fails even after a
 * diagonal shift of 1e-10 of its trace). */
int flr_set_variance_mode(flr_ctx *ctx, int32_t mode);

/* Allocate a neighbour list for systems of up to n_atoms atoms (device
 * memory: n_atoms * max_nbr * 4 bytes plus O(n_atoms) bookkeeping). */
int flr_nbrlist_create(flr_ctx *ctx, int32_t n_atoms, flr_nbrlist **out);
int flr_nbrlist_destroy(flr_nbrlist *nl);

/* Device views of a built list: entries[n][max_nbr] int32 =
 * (j << 8) | (s_j << 7) | image code, with s_j the species of atom j (0 or 1)
 * and code = (sx+2)*25 + (sy+2)*5 + (sz+2) for the lattice image
 * S = (sx, sy, sz) of atom j; count[n] int32 neighbours per row;
 * group[n] int32 compaction class (-1: no neighbours).  Lists hold fewer
 * than 2^24 atoms. */
int flr_nbrlist_view(const flr_nbrlist *nl, int32_t **entries, int32_t **count, int32_t **group,
                     int32_t *max_nbr);

/* Cell-list neighbour search (Sec. V-C neighbour lists; Sec. V-B local
 * environment): every (i, j, S) with |r_j + S.cell - r_i| < r_cut + skin,
 * (j, S) != (i, 0), rows ordered by visiting bins in a fixed stencil
 * order and atoms inside a bin by index.  Distances are decided in FP32,
 * and in FP64 within 1e-5 relative of the cutoff.  Also classifies every
 * atom for the species-block compaction and records the positions for the
 * displacement trigger.  SYNCHRONIZES the stream (the bin grid is planned
 * from the atoms' bounding box).  FLR_ENBR_OVERFLOW if a row exceeds
 * max_nbr (the message gives the count needed). */
int flr_build_neighbors(flr_ctx *ctx, const flr_system *sys, flr_nbrlist *nl, flr_stream_t stream);

/* Neighbour lists of every structure of a batch at once (same rules as
 * flr_build_neighbors, each structure with its own cell; rows refer to
 * batch-wide atom indices).  The list must have capacity for n_atoms.
 * SYNCHRONIZES the stream once (the bin grids are planned from the
 * structures' bounding boxes). */
int flr_build_neighbors_batch(flr_ctx *ctx, const flr_batch *batch, flr_nbrlist *nl, flr_stream_t stream);

/* Energy, forces and uncertainty of every atom of a batch in one launch
 * sequence (Eq. 1, Eq. 2; used for serving and for batched
 * differentiation).  Per-atom outputs cover all atoms of the batch; when
 * out->totals is not NULL it is a device double[n_structs][FLR_NTOTALS] and
 * receives each structure's totals (FP64 energy and virial, max sigma,
 * isolated atoms), each reduced in a fixed order.  Asynchronous. */
int flr_energy_forces_uncertainty_batch(flr_ctx *ctx, const flr_batch *batch, const flr_nbrlist *nl,
                                        flr_outputs *out, flr_stream_t stream);

/* Backward pass of the energy (differentiation of Eq. 1) for a batch whose
 * list was built by flr_build_neighbors(_batch): for the loss
 * L = sum_i u_i E_i with u = grad_energy (device float[n_atoms]),
 *   grad_pos  = dL/dr  (device float[n_atoms][3]) = -(forces of the weighted energy),
 *   grad_beta = dL/dbeta_s = sum over atoms i of species s of u_i d_i d_i^T
 *               (device float[n_species][d_full][d_full], overwritten; may be NULL).
 * The descriptors, basis values and quadratic forms are recomputed (the
 * basis is re-evaluated per pair inside the force kernel), so nothing is
 * stored between the forward and the backward call.  Asynchronous. */
int flr_energy_backward(flr_ctx *ctx, const flr_batch *batch, const flr_nbrlist *nl, const float *grad_energy,
                        float *grad_pos, float *grad_beta, flr_stream_t stream);

/* Normalized ACE-B2 descriptors d = B / ||B|| in the full layout
 * (Sec. V-B): d_hat device float[n][d_full] (components outside an atom's
 * compaction block are written as 0), norm device float[n] = ||B||. */
int flr_compute_descriptors(flr_ctx *ctx, const flr_system *sys, const flr_nbrlist *nl,
                            float *d_hat, float *norm, flr_stream_t stream);

/* Energy, forces and uncertainty of every atom (Eq. 1, Eq. 2, Sec. V-B
 * force reordering): descriptor -> quadratic forms on the selected
 * precision -> reordered force back-propagation with a deterministic
 * fixed-point scatter -> FP64 reductions.  Asynchronous. */
int flr_energy_forces_uncertainty(flr_ctx *ctx, const flr_system *sys, const flr_nbrlist *nl,
                                  flr_outputs *out, flr_stream_t stream);

/* n_steps of velocity-Verlet MD (metal units): half kick, drift, neighbour
 * rebuild when due (every rebuild_every steps, or when an atom moved more
 * than skin/2 since the last build, decided on the device), forces, half
 * kick.  Positions are wrapped into the cell at each rebuild.  The list
 * must have been built once with flr_build_neighbors.  With a thermostat
 * (st->temperature > 0), Nose-Hoover half steps wrap each step: xi is
 * advanced from the kinetic energy and the velocities are scaled by
 * exp(-xi dt / 2).  Asynchronous, except that the call synchronizes the
 * stream at its end when the thermostat is on (xi and eta return to *st)
 * and after every step when sigma_stop > 0 (the stop test reads a count). */
int flr_md_step(flr_ctx *ctx, flr_md_state *st, flr_nbrlist *nl, int32_t n_steps,
                flr_outputs *out, flr_stream_t stream);

/* Host copies of the MD state and of a step's results for flr_md_step_host.
 * All are HOST arrays (page-locked memory gives full copy speed; pageable
 * memory works but the copies then stage through the driver).  pos and vel
 * are float[n][3] (x, y, z), read before each step and overwritten with the
 * state after it.  energy (float[n]), forces (float[n][3]), variance
 * (float[n]), sigma (float[n]) and totals (double[FLR_NTOTALS]) may each be
 * NULL; those given receive the results of the call's last step.  The
 * caller owns every array. */
typedef struct {
    float *pos;
    float *vel;
    float *energy;
    float *forces;
    float *variance;
    float *sigma;
    double *totals;
} flr_host_state;

/* flr_md_step with the MD state kept in host memory (the production loop of
 * Sec. VI-A with the integrator's positions and velocities owned by the
 * caller).  Each of n_steps copies host->pos and host->vel to the device
 * (st->pos and st->vel, device float[n][4], are the working copies: their
 * x, y, z are overwritten and w is set to 0), runs one flr_md_step and
 * copies the new positions and velocities back; after the last step the
 * requested results follow.  st and out are as for flr_md_step (forces
 * must stay the same device buffer from call to call while forces_valid is
 * set).
 * Asynchronous: the copies run on two copy streams of the context, in eight
 * chunks, each chunk's upload for the next step starting once its download
 * has landed.  A step's positions are final after its drift and list
 * rebuild and are downloaded then, while its kernels run, so only the
 * velocities' round trip lies between two steps; the results read-back of
 * one call overlaps the next call's kernels (a call's quadratic forms wait
 * for the previous call's read-back before they overwrite the outputs).  The host arrays may be
 * read or changed only after flr_sync or after `stream` has passed
 * flr_host_join.  FLR_EINVAL for NULL pos or vel or the conditions of
 * flr_md_step. */
int flr_md_step_host(flr_ctx *ctx, flr_md_state *st, flr_nbrlist *nl, int32_t n_steps, flr_outputs *out,
                     const flr_host_state *host, flr_stream_t stream);

/* Make `stream` wait (on the device, without blocking the host) until every
 * copy that flr_md_step_host has enqueued on this context has landed. */
int flr_host_join(flr_ctx *ctx, flr_stream_t stream);

/* Synchronize `stream` (and the context's host-copy streams, if
 * flr_md_step_host has created them) and report (and clear) device-side
 * errors. */
int flr_sync(flr_ctx *ctx, flr_stream_t stream);

/* Number of kernels the library launched on this context so far, as counted
 * on the host.  flr_md_step runs each step's list rebuild as a conditional
 * graph: it counts the graph's one condition kernel per step, and the
 * FLR_REBUILD_KERNELS kernels of a rebuild run only on the steps that
 * rebuild (FLR_TOT_N_REBUILDS of them), which the host cannot see. */
#define FLR_REBUILD_KERNELS 13
int64_t flr_launch_count(const flr_ctx *ctx);

/* Cell-list neighbour search that allocates no memory.  (No counterpart in
 * the paper: this is a deployment variant of flr_build_neighbors.)
 *
 * For callers that cannot call cudaMalloc: a process whose device memory is
 * fixed at start-up (a serving process that reserves its whole budget once,
 * or a host framework that owns every device allocation through its own
 * pool), or a caller that holds no flr_ctx.  Inputs and outputs are the
 * caller's: sys (as for flr_build_neighbors), r_list = list cutoff
 * (r_cut + skin, A), max_nbr (multiple of 32 in [32, 512]), entries: device
 * int32[n][max_nbr] and count: device int32[n], in the format of
 * flr_nbrlist_view.  Rows hold the same pairs in the same order as
 * flr_build_neighbors with r_cut + skin = r_list.
 *
 * Every other buffer lives in one fixed device array inside the library
 * (about 3.9 MB, held by every GPU that loads the library until the process
 * exits), so the sizes are bounded: at most 65,536 atoms and 65,536 cell-list
 * bins; larger inputs return FLR_EINVAL with a message naming the limit.
 * The first call on a device looks up the array's device address with that
 * device current (make that first call before any stream capture).  All
 * calls share the array, so calls whose GPU work overlaps (several host
 * threads, or several streams) race; serialize them.  The call synchronizes
 * the stream twice (bounding box, then status) and returns
 * FLR_ENBR_OVERFLOW when a row exceeds max_nbr. */
int flr_build_neighbors_noalloc(const flr_system *sys, double r_list, int32_t max_nbr, int32_t *entries,
                                int32_t *count, flr_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching evaluation loop.  (No counterpart in the
 * paper, whose structures run one per MD job; each request is evaluated by
 * the same calls as flr_energy_forces_uncertainty_batch, Eq. 1 and Eq. 2
 * per atom, so a request's per-atom results do not depend on what else
 * shares its batch.)
 *
 * A server owns one worker thread and two batch slots on the context's
 * device; each slot has its own CUDA stream, pinned host arena, device
 * input/output arrays and neighbour list.  flr_server_submit() queues a
 * request (host inputs, host outputs) and returns at once.  The worker takes
 * queued requests in arrival order into a free slot while the batch's device
 * memory stays within the budget (and within max_batch_structs /
 * max_batch_atoms), packs them into the slot's pinned arena, and enqueues on
 * the slot's stream: one host-to-device copy per array, the bin-grid plan
 * (made on the host, no mid-batch synchronization), the neighbour build,
 * the evaluation, one device-to-host copy per array.  The two slots' batches
 * overlap on the device: one batch's copies and neighbour build run while
 * the other batch is evaluated.  Evaluations themselves run one at a time
 * (they share the context's workspace).  When a batch's copies are done the
 * worker writes each request's output arrays and reports the completions,
 * which are collected with flr_server_poll().
 *
 * While a server exists its worker is the only user of the context: make no
 * other call on that context (or its neighbour lists) until
 * flr_server_destroy() returns.
 * ------------------------------------------------------------------------ */
typedef struct flr_server flr_server;

typedef struct {
    size_t hbm_budget_bytes;     /* device memory the batches may use (workspace, neighbour list, I/O);
                                    the model tables (a few MB) are outside it */
    int32_t max_batch_structs;   /* <= 0: no limit besides memory */
    int32_t max_batch_atoms;     /* <= 0: no limit besides memory */
    int64_t reserve_atoms;       /* > 0: allocate device and pinned memory for batches of this many
                                    atoms at creation, so no batch up to this size allocates;
                                    0: grow on demand (doubling, synchronizes the device) */
    int32_t reserve_structs;     /* structures per batch reserved with reserve_atoms (>= 1) */
} flr_server_params;

/* One structure to evaluate.  Inputs are host arrays read during
 * flr_server_submit() (copied; they may be reused when it returns).
 * Outputs are host arrays written by the worker before the request's
 * completion is reported; they must stay valid until then.  Any output
 * may be NULL. */
typedef struct {
    int32_t n_atoms;
    const float *pos;            /* host float[n][4] (x, y, z, unused) */
    const int32_t *species;      /* host int32[n] */
    double cell[9];              /* rows are lattice vectors */
    int32_t pbc[3];
    float *energy;               /* host float[n] */
    float *forces;               /* host float[n][3] */
    float *variance;             /* host float[n] */
    float *sigma;                /* host float[n] */
    double *totals;              /* host double[FLR_NTOTALS] */
    uint64_t tag;                /* returned in the completion */
} flr_request;

typedef struct {
    uint64_t tag;
    int32_t status;              /* FLR_OK, or the error of the batch that held the request */
    int32_t batch_structs;       /* structures in that batch */
    int64_t batch_atoms;         /* atoms in that batch */
    int64_t t_submit_ns;         /* steady-clock times: submitted, batch enqueued on the GPU, */
    int64_t t_start_ns;          /* outputs written */
    int64_t t_done_ns;
    int32_t slot;                /* batch slot that ran the request (0 or 1) */
    /* device timestamps of the request's batch (ms since the server was
     * created, from CUDA events on the slot's stream): copies started,
     * neighbour build done, evaluation started (after the previous batch's
     * evaluation), evaluation done, outputs copied back */
    float gpu_start_ms, gpu_built_ms, gpu_eval_start_ms, gpu_eval_end_ms, gpu_done_ms;
} flr_completion;

typedef struct {
    int64_t requests;            /* completed requests */
    int64_t batches;
    int64_t atoms;               /* atoms evaluated */
    int64_t max_batch_atoms_seen;
    int64_t queued;              /* requests waiting now */
    int64_t reserved_bytes;      /* device memory the server holds now */
    int64_t bytes_per_atom;      /* admission cost of one atom */
    char last_error[256];        /* message of the last failed batch ("" if none) */
    int64_t batches_overlapped;  /* batches enqueued while the other slot's batch was in flight */
    int64_t grow_events;         /* times device memory had to grow under load (each synchronizes) */
    double grow_ms, pack_ms, enqueue_ms, finish_ms;   /* worker host time: growing, packing inputs,
                                                         enqueueing, writing outputs (ms, summed) */
} flr_server_stats;

/* Device bytes one atom of a batch costs: the context's workspace once, and
 * a neighbour-list row and the I/O arrays for each of the server's two
 * slots; the figure the admission check multiplies by the atom count. */
int flr_bytes_per_atom(const flr_ctx *ctx, int64_t *bytes);

/* Start a server on ctx (the model must be set).  FLR_EBUDGET if the budget
 * cannot hold a single atom or the reservation.  With reserve_atoms > 0 the
 * call allocates the reservation (device and pinned host memory) before it
 * returns. */
int flr_server_create(flr_ctx *ctx, const flr_server_params *params, flr_server **out);

/* Queue one request (thread-safe).  FLR_EBUDGET if the request alone
 * exceeds the budget or max_batch_atoms; FLR_EINVAL for invalid input. */
int flr_server_submit(flr_server *srv, const flr_request *req);

/* Collect up to max finished requests into out[0 .. *n_out - 1], waiting up
 * to wait_seconds for the first one (0: do not wait). */
int flr_server_poll(flr_server *srv, flr_completion *out, int32_t max, int32_t *n_out, double wait_seconds);

int flr_server_stats_read(flr_server *srv, flr_server_stats *stats);

/* Stop the worker after the batches in flight and free the server.
 * Requests still queued are dropped without a completion. */
int flr_server_destroy(flr_server *srv);

/* Measured FP32 FMA throughput of `device` (no counterpart in the paper: the
 * roofline denominator of the descriptor and force kernels, which are bound
 * by FP32 arithmetic).  Runs one warm-up and then `launches` launches of a
 * kernel in which every thread advances 8 independent register-resident FMA
 * chains, on every SM (SM count read from the device) at its occupancy
 * limit, each launch timed with CUDA events.  Returns the best and the
 * median rate in TFLOP/s (2 flop per FMA) and the SM count.  Allocates and
 * frees a few bytes of device memory; synchronous; leaves `device` current. */
int flr_fp32_fma_peak(int device, int32_t launches, double *tflops_best, double *tflops_median, int32_t *num_sms);

/* Kernel classes of flr_profile_read. */
#define FLR_KERNEL_DESCRIPTOR 0   /* A, B2, normalization (one launch per evaluation) */
#define FLR_KERNEL_QFORM 1        /* quadratic-form GEMM (SIMT or tcgen05) */
#define FLR_KERNEL_FORCE 2        /* E, V, sigma, reordered back-propagation, per-pair forces */
#define FLR_KERNEL_FINALIZE 3     /* fixed point -> forces, half kick, FP64 totals */
#define FLR_KERNEL_DRIFT 4        /* MD half kick + drift + displacement check */
#define FLR_KERNEL_REBUILD 5      /* the (conditional) neighbour rebuild sequence */
#define FLR_KERNEL_FUSED 6        /* fused one-species descriptor + quadratic forms (FLR_OPT_FUSED_ONE_SPECIES) */
#define FLR_KERNEL_CLASSES 7

/* Per-kernel device timing: when on, every launch of the classes above is
 * bracketed by CUDA events recorded on its own stream (off by default;
 * turning it on clears the accumulated totals). */
int flr_profile_enable(flr_ctx *ctx, int32_t on);

/* Accumulated device time (ms) and launch count of one kernel class since
 * profiling was enabled.  Waits for the recorded events. */
int flr_profile_read(flr_ctx *ctx, int32_t kernel_class, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* FLARE_GB_H */
