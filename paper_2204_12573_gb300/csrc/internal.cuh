// Internal declarations shared by the translation units of libflare_gb.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>

#include "../../include/flare_gb.h"

namespace flr {

constexpr int kSpecies = 2;        // species handled by the device code
constexpr int kL = 3;              // l_max handled by the device code
constexpr int kNLM = (kL + 1) * (kL + 1);   // 16 real harmonics
constexpr int kGroups = kSpecies * 3;        // (central species) x (class: both, only 0, only 1)
constexpr int kWarpsDesc = 8;      // warps per CTA of the per-atom kernels

// device status word bits
enum : int {
    kErrOverflow = 1,
    kErrNonFinite = 2,
    kErrShift = 4,
    kErrTimeout = 8,
    kErrSpecies = 16,
};

// Group g = s_center * 3 + cls; cls 0 uses the full descriptor, cls 1 + t
// the one-species block of species t.
__host__ __device__ inline int group_cls(int g) { return g % 3; }
__host__ __device__ inline int group_species(int g) { return g / 3; }
__host__ __device__ inline bool group_full(int g) { return (g % 3) == 0; }

// Region of the compact descriptor rows: 0 = full (d_full), 1 = single (d_single).
__host__ __device__ inline int group_region(int g) { return group_full(g) ? 0 : 1; }

struct Dims {
    int N;            // n_max
    int C;            // S * N channels
    int nA;           // C * 16 entries of A
    int d_full, d_single;
    int kp32[2];      // K padded to 32 (FP32 / TF32 rows), per region
    int kp64[2];      // K padded to 64 (BF16 rows), per region
    int K[2];         // unpadded K per region
    int nrows_pad[2]; // rows of the B operand (2K padded to a multiple of 288)
};

// Device-side group table, filled by the group-partition kernel.
struct GroupTab {
    int count[kGroups];
    int off[kGroups];       // first row inside its region
    int tiles_simt[kGroups + 1];  // prefix of SIMT tiles (M-tiles x N-tiles)
    int tiles_tc[kGroups + 1];    // prefix of tensor-core M-tiles (each covers all its column chunks)
    int n_isolated;         // atoms with an empty list
    int max_count;          // longest overflowing neighbour row (before clipping); 0 without overflow
};

struct Plan {
    int nb[3];          // bins per lattice direction
    int R[3];           // stencil reach in bins
    float flo[3];       // lower fractional bound of the bin grid (0 along periodic dirs)
    float fspan[3];     // fractional span of the bin grid (1 along periodic dirs)
    double bscale[3];   // nb / fspan in FP64 (bin coordinate = (frac - flo) * bscale)
    double cell[9];
    double inv[9];      // inverse of the cell matrix (frac = pos . inv)
    float invf[9];      // inv rounded to FP32 (the in-bin offsets used to prune the stencil)
    int pbc[3];
    long long nbins;
    long long bin_base; // first global bin of this structure in a batch
    float bw[3];        // bin width along each direction's plane normal (A)
    int orth;           // 1: orthogonal cell (box distances are exact Euclidean distances)
};

}  // namespace flr

struct flr_nbrlist {
    flr_ctx *ctx;
    int n_cap;
    int n;                 // atoms of the last build
    int max_nbr;
    int32_t *entries;      // [n_cap][max_nbr]
    int32_t *count;        // [n_cap]
    int32_t *group;        // [n_cap]
    int32_t *row;          // [n_cap] row inside the group's region
    int32_t *atom_of_row;  // [2][n_cap]
    float4 *pair_rec;      // [n_cap][max_nbr] pairs inside r_cut of the last descriptor pass:
                           // (r_ij, j | s_j << 25), written by k_desc, read by k_force
    int32_t *pair_cnt;     // [n_cap] pairs inside r_cut
    float4 *pos_ref;       // positions at the last build
    int32_t *img;          // [n_cap] packed image offset of the wrapped position
    int32_t *atom_bin;     // [n_cap]
    int32_t *bin_atoms;    // [n_cap]
    float4 *pos_bin;       // [n_cap] positions in bin order, species bits in .w (list build only)
    int32_t *bin_start;    // [nbins_cap + 1]
    int32_t *bin_fill;     // [nbins_cap]
    int32_t *blk_group;    // [n_blocks][8] per-block group counts
    flr::GroupTab *gtab;   // device
    int32_t *flags;        // device [4]: [0] rebuild needed, [1] rebuild counter
    int *status;           // device status word the list build reports into (the context's by default)
    int *sched;            // device work counter of the list build (one of the context's by default)
    float *bbox;           // device [structs_cap][8] fractional min / max
    long long nbins_cap;
    flr::Plan plan;        // structure 0 (the single-structure calls)
    bool planned;
    // batches of structures: atoms of structure s are [offsets[s], offsets[s+1])
    int n_structs;
    int structs_cap;
    int32_t *struct_of;    // device [n_cap] structure of each atom (nullptr when n_structs == 1)
    int32_t *offsets_d;    // device [structs_cap + 1]
    float4 *shift_d;       // device [structs_cap][125][2] image shifts S.cell, FP32 hi and lo
    flr::Plan *plans_d;    // device [structs_cap]
    flr::Plan *plans_h;    // host  [structs_cap]
    int32_t *offsets_h;    // host  [structs_cap + 1]
    long long nbins_total; // bins of all structures
    void *rgraph;          // the MD steps' conditional rebuild graph (nbr.cu), or nullptr
};

// TMA tensor maps of the tcgen05 path: A operands per region (BF16 hi / lo,
// or FP32 rows for TF32) and B operands per group.
struct TcMaps {
    CUtensorMap a[2][2];
    CUtensorMap b[flr::kGroups][2];
};

struct flr_ctx {
    flr_params p;
    int device;
    int num_sms;
    flr::Dims dims;
    int *status;               // device status word [4]
    long long launches;
    // model, per group
    bool model_set[flr::kSpecies];
    double *beta_h[flr::kSpecies];     // host copies (symmetrized), d_full^2
    double *sigma_h[flr::kSpecies];
    int var_mode;                      // FLR_VAR_*
    int var_factored[flr::kGroups];    // 1: the group's Sigma rows hold L^T (V = |L^T d|^2)
    double *S64[flr::kGroups];         // FP64 Sigma block of each group (K x K), for the FP64 variance
    float sigma_norm[flr::kGroups];    // largest eigenvalue of each group's Sigma block (power iteration)
    int32_t *ref_list;                 // [ws_n] atoms queued for the FP64 variance
    int *ref_count;                    // device counter of ref_list
    int *sched;                        // device work counters [8]: descriptor, force (two-species), list build, force (one-species), one-species quadratic-form tiles
    double *md_sc;                     // MD scalars: [0] xi, [1] eta, [2] KE, [3] scale, [8..8+256) KE partials
    double *md_totals;                 // totals of flr_md_step when the caller passes none
    int *md_cnt;                       // [2] uncertainty and coordination counts
    float *W32[flr::kGroups];          // [nrows_pad][kp32]  B operand rows (beta rows, then Sigma rows)
    __nv_bfloat16 *Whi[flr::kGroups];  // [nrows_pad][kp64]
    __nv_bfloat16 *Wlo[flr::kGroups];
    float *Wtf[flr::kGroups];          // [nrows_pad][kp32]  W32 rounded to nearest TF32 (TF32 B operand)
    // index tables (device): packed (a | b << 8 | l << 16) for each compact component
    int32_t *tab_full;
    int32_t *tab_single;
    // workspace
    int ws_n;                  // atoms the workspace is sized for
    float *A;                  // [n][nA]
    float *norm;               // [n]
    float *D32[2];             // [n][kp32[r]]
    __nv_bfloat16 *Dhi[2];     // [n][kp64[r]]
    __nv_bfloat16 *Dlo[2];
    float *Dtf[2];             // [n][kp32[r]] descriptor rows rounded to nearest TF32 (TF32 A operand;
                               // allocated on first TF32 use, sized like D32)
    float *P[2];               // [n][2K[r]] quadratic-form products (FP32 SIMT path only)
    float *G[2];               // [n][K[r]]  g = dE/dB rows, consumed by the force kernel
    long long *Facc;           // [n][3] fixed point
    float *vir_atom;           // [n][9] per-atom virial (batches)
    float *scratch_out;        // [3][n] E, V, sigma of the backward pass
    double *partials;          // [n_blocks][16]
    int n_part;
    void *fmaps;               // tensor maps of the fused one-species kernel (built once per context)
    void *q1maps;              // tensor maps of the one-species quadratic-form kernel
    int q1maps_n;              // workspace size they were encoded for
    int use_fused;             // FLR_OPT_FUSED_ONE_SPECIES
    int overlap;               // FLR_OPT_OVERLAP_TWO_SPECIES
    TcMaps *maps;              // host copy of the current tensor maps
    int maps_n;                // workspace size the maps were encoded for
    int maps_prec;
    // per-kernel event timing (flr_profile_*)
    struct ProfState *prof;
    // host-state MD (flr_md_step_host): copy streams, events and staging rows (api.cu)
    struct HostIO *hio;
    cudaEvent_t out_gate;      // when set, evaluations wait for it before writing their outputs
};

struct ProfState {
    struct Rec {
        cudaEvent_t a, b;
        int cls;
    };
    bool on;
    Rec *recs;
    int n_recs, cap;
    cudaEvent_t *pool;
    int n_pool, pool_cap;
    double ms[FLR_KERNEL_CLASSES];
    long long count[FLR_KERNEL_CLASSES];
};

namespace flr {
// Bracket a launch with events when profiling is on (no-ops otherwise).
void prof_begin(flr_ctx *ctx, int cls, cudaStream_t st);
void prof_end(flr_ctx *ctx, int cls, cudaStream_t st);
}  // namespace flr

namespace flr {

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
inline void count_launch(flr_ctx *ctx, int k = 1) { ctx->launches += k; }

// ---- launchers (one per translation unit) ----
int launch_rebuild(flr_ctx *ctx, flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                   cudaStream_t st, bool wrap_positions, float4 *pos_mut);
// host_bb: per-structure fractional bounding boxes float[n_structs][8]
// computed on the host (host_frac_bbox); nullptr: computed on the device,
// which synchronizes the stream once.
int plan_batch(flr_ctx *ctx, flr_nbrlist *nl, int n_structs, const int32_t *offsets, const double *cells,
               const int32_t *pbc, const float4 *pos, int n, cudaStream_t st, const float *host_bb = nullptr);
void host_frac_bbox(const double *cell, const float *pos4, int n, float bb[8]);
int launch_set_rebuild(flr_ctx *ctx, flr_nbrlist *nl, cudaStream_t st);
// The rebuild sequence of launch_rebuild as the body of a conditional graph
// node that runs only when the list's rebuild flag is set (MD steps): a step
// that needs no rebuild then launches one small kernel instead of the whole
// early-exiting sequence.  The graph is kept with the list and rebuilt when
// any host-side argument of the sequence changes.
int launch_rebuild_cond(flr_ctx *ctx, flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                        cudaStream_t st, bool wrap_positions, float4 *pos_mut);
void free_rebuild_graph(flr_nbrlist *nl);
// serving-loop access to the context (api.cu)
int srv_reserve_workspace(flr_ctx *ctx, int n);
int srv_evaluate(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, double *seg_totals, cudaStream_t st);
int srv_status_code(int st);
int srv_check_model(const flr_ctx *ctx);
void bytes_per_atom_parts(const flr_ctx *ctx, int64_t *workspace, int64_t *slot);
// grow a list's per-structure tables and bin arrays ahead of use (so that
// planning batches of up to n_structs structures and nbins bins allocates nothing)
int nbrlist_reserve_batch(flr_ctx *ctx, flr_nbrlist *nl, int n_structs, long long nbins);
// Descriptor kernel over atoms 0 .. n-1, or over order[0 .. m) with m read on
// the device as *n_dev0 (+ *n_dev1), capped at n.
int launch_desc(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                cudaStream_t st, const int32_t *order = nullptr, const int *n_dev0 = nullptr,
                const int *n_dev1 = nullptr, bool skip_d32_one = false);
int launch_expand_desc(flr_ctx *ctx, const flr_nbrlist *nl, int n, float *d_hat, float *norm,
                       cudaStream_t st);
int launch_qform_simt(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st);
// only_full: take only the tiles of the two-species (full-descriptor) groups
int launch_qform_tc(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st, bool only_full = false);
int encode_tile_map(CUtensorMap *m, const void *ptr, bool bf16, int cols, int rows, int box_cols, int box_rows,
                    int swizzle_bytes);
// The fused one-species kernel (descriptor -> tensor-core quadratic forms ->
// E, V, sigma, g rows) over the one-species compaction groups; false from
// fused_eligible when the context cannot take it (precision, compaction, N).
bool fused_eligible(const flr_ctx *ctx);
int launch_fused(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, cudaStream_t st);
void free_fused_maps(flr_ctx *ctx);
// Quadratic forms of the one-species tiles, 3xBF16 (each tile's A hi/lo
// resident in shared memory; tiles past the first per CTA claimed from a counter)
// pdl: launched as a programmatic dependent of the kernel before it on st
// (which must trigger its dependents); its tile counter (sched[4]) must have
// been cleared on st before that kernel
int launch_qform1(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st, bool pdl);
void free_q1_maps(flr_ctx *ctx);
int launch_force(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, float *vir_atom, const float *weight, cudaStream_t st);
int launch_seg_totals(flr_ctx *ctx, const flr_nbrlist *nl, const flr_outputs *out, const float *vir_atom,
                      double *totals, cudaStream_t st);
struct KickArgs {
    float4 *vel;
    const int *species;
    float half_dt_over_m[kSpecies];   // (dt/2) * FTM2V / m_s
    float half_m[kSpecies];            // m_s / 2 / FTM2V  (kinetic energy in eV from A/ps)
    int enabled;
    const double *scale;               // thermostat velocity scale before the first kick (drift), or nullptr
};
int launch_finalize(flr_ctx *ctx, const flr_nbrlist *nl, int n, flr_outputs *out, const KickArgs &kick, float sign,
                    cudaStream_t st);
int launch_dbeta(flr_ctx *ctx, const flr_nbrlist *nl, const float *u, float *grad_beta, cudaStream_t st);
// MD extras (md.cu): kinetic energy, Nose-Hoover half step, velocity scaling,
// uncertainty and coordination counts
int launch_kinetic(flr_ctx *ctx, const float4 *vel, const int32_t *species, int n, const double *masses,
                   double *part, double *ke, cudaStream_t st);
int launch_thermo_half(flr_ctx *ctx, double *sc, const double *ke_in, double gkT, double Q, double dt, double *totals,
                       cudaStream_t st);
int launch_scale_vel(flr_ctx *ctx, float4 *vel, int n, const double *scale, cudaStream_t st);
int launch_count_above(flr_ctx *ctx, const float *sigma, int n, float thr, int *count, double *totals,
                       cudaStream_t st);
int launch_cn_count(flr_ctx *ctx, const flr_nbrlist *nl, const int32_t *species, int n, int cs, float rc,
                    int *count, double *totals, cudaStream_t st);
// FP64 re-evaluation of the variance of the atoms the epilogue queued (FLR_VAR_AUTO)
int launch_variance_fp64(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st);
constexpr float kVarCancel = 32.f;   // queue an atom when V < (sum_k |d_k (Sigma d)_k|) / kVarCancel
// ... or when V < kVarSmall * |Sigma_c|_2: the FP32 GEMM's absolute error on V scales with
// |Sigma_c|_2, so a variance this small relative to the prior's scale keeps too few digits
// (the GEMM's own cancellation, which the final sum cannot see).  Per precision:
constexpr float kVarSmallFP32 = 2e-3f;
constexpr float kVarSmallBF16x3 = 2e-2f;
int launch_md_drift(flr_ctx *ctx, flr_nbrlist *nl, float4 *pos, float4 *vel, const float *forces,
                    const int *species, int n, const KickArgs &kick, float dt, float disp2_max,
                    cudaStream_t st);
// MD state between host float[n][3] staging rows and the device float[n][4]
// working copies (flr_md_step_host)
int launch_state_unpack(flr_ctx *ctx, const float *pos3, const float *vel3, float4 *pos, float4 *vel, int n,
                        cudaStream_t st);
int launch_state_pack(flr_ctx *ctx, const float4 *src, float *dst3, int n, cudaStream_t st);

// Grid of a persistent kernel: every SM filled to its occupancy limit, but
// never more blocks than there is work for.
template <typename K>
inline int persistent_grid(K kernel, int threads, int num_sms, long long work_blocks)
{
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * num_sms;
    if (work_blocks < g) g = work_blocks;
    return (int)(g < 1 ? 1 : g);
}
constexpr int kMaxPartials = 8192;   // rows of the reduction partials buffers

// Dynamic work distribution for the per-atom kernels: a warp takes CH
// consecutive positions of a work sequence at a time from a global counter
// (zeroed before the launch) and claims its next chunk one chunk ahead, so
// the item after the current one is always known and can be prefetched.
// Warps that run into expensive items (two-species environments, surface
// layers, dense bins) take fewer chunks, so the kernel ends when the work
// does instead of when the slowest fixed block does.
constexpr int kWarpChunk = 16;   // atoms per chunk in the force kernel
template <int CH>
struct WarpChunksT {
    int n, nchunks, cur, nxt, k;
    int *counter;
    __device__ __forceinline__ void init(int *ctr, int n_, int lane)
    {
        counter = ctr;
        n = n_;
        nchunks = (n_ + CH - 1) / CH;
        k = 0;
        int c0 = 0, c1 = 0;
        if (lane == 0) {
            c0 = atomicAdd(ctr, 1);
            c1 = atomicAdd(ctr, 1);
        }
        cur = __shfl_sync(0xffffffffu, c0, 0);
        nxt = __shfl_sync(0xffffffffu, c1, 0);
    }
    // sequence position of the current item (n when the warp is done)
    __device__ __forceinline__ int pos() const { return cur < nchunks ? cur * CH + k : n; }
    // the position after the current one
    __device__ __forceinline__ int peek() const
    {
        if (cur >= nchunks) return n;
        const int p = cur * CH + k + 1;
        if (k + 1 < CH && p < n) return p;
        return nxt < nchunks ? nxt * CH : n;
    }
    // move to peek(); the whole warp calls it
    __device__ __forceinline__ void advance(int lane)
    {
        const int p = cur * CH + k + 1;
        if (cur < nchunks && k + 1 < CH && p < n) {
            ++k;
            return;
        }
        cur = nxt;
        k = 0;
        int c = nchunks;
        if (lane == 0 && cur < nchunks) c = atomicAdd(counter, 1);
        nxt = __shfl_sync(0xffffffffu, c, 0);
    }
};
using WarpChunks = WarpChunksT<kWarpChunk>;

// The same claims with the chunk length chosen at launch: a launch over few
// atoms (the two-species rows of a mostly one-species system) takes them one
// by one, so they spread over all warps instead of 16 to a warp.
struct WarpChunksR {
    int n, ch, nchunks, cur, nxt, k;
    int *counter;
    __device__ __forceinline__ void init(int *ctr, int n_, int ch_, int lane)
    {
        counter = ctr;
        n = n_;
        ch = ch_;
        nchunks = (n_ + ch_ - 1) / ch_;
        k = 0;
        int c0 = 0, c1 = 0;
        if (lane == 0) {
            c0 = atomicAdd(ctr, 1);
            c1 = atomicAdd(ctr, 1);
        }
        cur = __shfl_sync(0xffffffffu, c0, 0);
        nxt = __shfl_sync(0xffffffffu, c1, 0);
    }
    __device__ __forceinline__ int pos() const { return cur < nchunks ? cur * ch + k : n; }
    __device__ __forceinline__ int peek() const
    {
        if (cur >= nchunks) return n;
        const int p = cur * ch + k + 1;
        if (k + 1 < ch && p < n) return p;
        return nxt < nchunks ? nxt * ch : n;
    }
    __device__ __forceinline__ void advance(int lane)
    {
        const int p = cur * ch + k + 1;
        if (cur < nchunks && k + 1 < ch && p < n) {
            ++k;
            return;
        }
        cur = nxt;
        k = 0;
        int c = nchunks;
        if (lane == 0 && cur < nchunks) c = atomicAdd(counter, 1);
        nxt = __shfl_sync(0xffffffffu, c, 0);
    }
};

// Tiles of 128 rows over the one-species compaction groups (1, 2, 4, 5), in
// that order: pre[k] is the first tile of the k-th of them.
struct OneTile {
    int g, row0, rend;
};
__device__ __forceinline__ int one_species_group(int k) { return k < 2 ? k + 1 : k + 2; }
__device__ __forceinline__ int one_species_tiles(const GroupTab &T, int pre[5])
{
    pre[0] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) pre[k + 1] = pre[k] + (T.count[one_species_group(k)] + 127) / 128;
    return pre[4];
}
__device__ __forceinline__ OneTile one_species_tile(const GroupTab &T, const int pre[5], int t)
{
    int k = 0;
    while (k < 3 && t >= pre[k + 1]) ++k;
    OneTile ti;
    ti.g = one_species_group(k);
    ti.row0 = T.off[ti.g] + (t - pre[k]) * 128;
    ti.rend = T.off[ti.g] + T.count[ti.g];
    return ti;
}

// ---- shared device helpers ----

// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits,
// ties away from zero), kept in FP32 storage with the low 13 bits zero.  The
// tensor core reads the top 19 bits of an FP32 operand, i.e. truncates; a
// value that is already TF32 passes through unchanged, so operands rounded
// here enter the product rounded to nearest instead of truncated.
__host__ __device__ inline uint32_t tf32_round_bits(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

// Decode a neighbour entry: (j << 8) | (s_j << 7) | code,
// code = (sx+2)*25 + (sy+2)*5 + (sz+2); s_j is the species of j (0 or 1).
__device__ __forceinline__ int entry_species(int e) { return (e >> 7) & 1; }
__device__ __forceinline__ int entry_atom(int e) { return (int)((unsigned)e >> 8); }
__device__ __forceinline__ int entry_code(int e) { return e & 127; }
constexpr int kCenterCode = 62;   // (0, 0, 0)

constexpr int kShiftCodes = 125;  // image codes (sx, sy, sz) in [-2, 2]^3

// Image shifts S.cell of the structure atom i belongs to: per structure and
// code, the FP64 shift split into FP32 hi and lo parts (two float4, .w unused),
// formed on the host from the cell rows (the lattice vectors).
struct Cells {
    const float4 *shift;       // [n_structs][kShiftCodes][2]
    const int32_t *struct_of;  // [n] or nullptr (one structure)
    __device__ __forceinline__ const float4 *of(int i) const
    {
        return shift + 2 * kShiftCodes * (struct_of ? __ldg(struct_of + i) : 0);
    }
};

// x_j - x_i + (th + tl) for one coordinate, in FP32 only: TwoSum (Knuth)
// gives x_j - x_i = s + e and s + th = u + f exactly, then the small terms
// are summed and added last.  The result is the FP32 rounding of the exact
// sum up to terms of relative size 2^-37, so a shift by a large lattice
// vector loses nothing to cancellation.
__device__ __forceinline__ float shifted_diff(float xj, float xi, float th, float tl)
{
    const float s = __fsub_rn(xj, xi);
    const float bs = __fsub_rn(s, xj);
    const float e = __fadd_rn(__fsub_rn(xj, __fsub_rn(s, bs)), __fsub_rn(-xi, bs));
    const float u = __fadd_rn(s, th);
    const float bu = __fsub_rn(u, s);
    const float f = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bu)), __fsub_rn(th, bu));
    return __fadd_rn(u, __fadd_rn(__fadd_rn(e, f), tl));
}

// Pair vector r_ij = r_j + S.cell - r_i in FP32 for the image code of a list
// entry.  Without an image shift the FP32 difference is correctly rounded;
// with one, see shifted_diff.
__device__ __forceinline__ float3 pair_vector(const float4 &pi, const float4 &pj, int code, const float4 *shift)
{
    if (code == kCenterCode) return make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z);
    const float4 hi = __ldg(shift + 2 * code), lo = __ldg(shift + 2 * code + 1);
    return make_float3(shifted_diff(pj.x, pi.x, hi.x, lo.x), shifted_diff(pj.y, pi.y, hi.y, lo.y),
                       shifted_diff(pj.z, pi.z, hi.z, lo.z));
}

}  // namespace flr
