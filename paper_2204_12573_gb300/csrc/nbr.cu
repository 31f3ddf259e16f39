// Cell-list neighbour search and species-block classification.
//
// The local environment of atom i is every (j, S) with
// |r_j + S.cell - r_i| < r_cut + skin (Sec. V-B "Local structure
// descriptors"; Sec. V-C: the list is built once and reused while atoms
// move less than half the skin).  Atoms are binned by fractional coordinate;
// each bin is at least (r_cut + skin) wide so a fixed stencil of bins covers
// every neighbour.  A batch of structures is handled in one pass: each
// structure has its own cell, bin grid (a contiguous range of global bins)
// and plan in device memory, and each atom knows its structure.  All steps
// run on the device; every kernel of the rebuild sequence first reads the
// list's "rebuild needed" flag and returns at once when it is clear, so an
// MD loop can enqueue the sequence every step and let the device decide.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace flr {
namespace {

constexpr int kScanBlock = 1024;
constexpr int kGroupBlock = 512;

__device__ __forceinline__ int ordered(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// Fractional coordinates, FP64 products and sums rounded one by one (no
// fused multiply-add), so host_frac_bbox reproduces them bit for bit.
__device__ __forceinline__ void frac_of(const float4 &p, const double *inv, double f[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d)
        f[d] = __dadd_rn(__dadd_rn(__dmul_rn((double)p.x, inv[d]), __dmul_rn((double)p.y, inv[3 + d])),
                         __dmul_rn((double)p.z, inv[6 + d]));
}

__device__ __forceinline__ int structure_of(const int32_t *struct_of, int i) { return struct_of ? struct_of[i] : 0; }

__global__ void k_bbox_init(int *bb, int n_structs)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 8 * n_structs; k += gridDim.x * blockDim.x) {
        const int d = k & 7;
        bb[k] = d < 3 ? ordered(FLT_MAX) : ordered(-FLT_MAX);
    }
}

// fractional bounding box of every structure (warp-reduced when a warp's
// atoms share a structure, which is the common case)
__global__ void k_bbox(const float4 *__restrict__ pos, int n, const Plan *plans, const int32_t *struct_of, int *bb)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n; base += warps * 32) {
        const int i = base + lane;
        const bool valid = i < n;
        const int s = valid ? structure_of(struct_of, i) : -1;
        float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        if (valid) {
            double f[3];
            frac_of(pos[i], plans[s].inv, f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lo[d] = (float)f[d];
                hi[d] = (float)f[d];
            }
        }
        const int s0 = __shfl_sync(0xffffffffu, s, 0);
        if (__all_sync(0xffffffffu, !valid || s == s0)) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                for (int o = 16; o; o >>= 1) {
                    lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                    hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
                }
            if (lane == 0)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    atomicMin(bb + 8 * s0 + d, ordered(lo[d]));
                    atomicMax(bb + 8 * s0 + 3 + d, ordered(hi[d]));
                }
        } else if (valid) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                atomicMin(bb + 8 * s + d, ordered(lo[d]));
                atomicMax(bb + 8 * s + 3 + d, ordered(hi[d]));
            }
        }
    }
}

__global__ void k_bbox_finish(int *bb, int n_structs)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 8 * n_structs; k += gridDim.x * blockDim.x)
        if ((k & 7) < 6) reinterpret_cast<float *>(bb)[k] = unordered(bb[k]);
}

// structure id of every atom from the batch offsets
__global__ void k_struct_of(const int32_t *offsets, int n_structs, int32_t *struct_of)
{
    for (int s = blockIdx.x; s < n_structs; s += gridDim.x)
        for (int i = offsets[s] + threadIdx.x; i < offsets[s + 1]; i += blockDim.x) struct_of[i] = s;
}

struct BinArgs {
    const float4 *pos;
    float4 *pos_mut;      // non-null: wrap positions in place (MD)
    int n;
    const Plan *plans;
    const int32_t *struct_of;
    int32_t *atom_bin, *img, *bin_count;
    float4 *pos_ref;
    GroupTab *gtab;
    const int32_t *flags;
    int *status;
};

__global__ void k_zero_bins(int32_t *cnt, long long nbins, const int32_t *flags)
{
    if (flags[0] == 0) return;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbins;
         b += (long long)gridDim.x * blockDim.x)
        cnt[b] = 0;
}

__global__ void k_bin(BinArgs a)
{
    if (a.flags[0] == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.gtab->max_count = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const Plan &P = a.plans[structure_of(a.struct_of, i)];
        float4 p = a.pos_mut ? a.pos_mut[i] : a.pos[i];
        double f[3];
        frac_of(p, P.inv, f);
        int im[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (P.pbc[d]) {
                im[d] = (int)floor(f[d]);
                f[d] -= im[d];
            }
        if (a.pos_mut && (im[0] | im[1] | im[2])) {
            // wrap in place: r -= img . cell, formed in FP64
            const double *c = P.cell;
            double x = (double)p.x - (im[0] * c[0] + im[1] * c[3] + im[2] * c[6]);
            double y = (double)p.y - (im[0] * c[1] + im[1] * c[4] + im[2] * c[7]);
            double z = (double)p.z - (im[0] * c[2] + im[1] * c[5] + im[2] * c[8]);
            p.x = (float)x;
            p.y = (float)y;
            p.z = (float)z;
            a.pos_mut[i] = p;
            im[0] = im[1] = im[2] = 0;
        }
        int b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // a product with the host's nb / fspan instead of an FP64 division per atom
            // (FP64 runs at a small fraction of the FP32 rate here)
            int k = (int)floor((f[d] - (double)P.flo[d]) * P.bscale[d]);
            b[d] = min(max(k, 0), P.nb[d] - 1);
            if (im[d] < -100 || im[d] > 100) atomicOr(a.status, kErrShift);
        }
        const int bin = (int)P.bin_base + (b[0] * P.nb[1] + b[1]) * P.nb[2] + b[2];
        a.atom_bin[i] = bin;
        a.img[i] = (im[0] & 0xFF) | ((im[1] & 0xFF) << 8) | ((im[2] & 0xFF) << 16);
        a.pos_ref[i] = p;
        atomicAdd(a.bin_count + bin, 1);
    }
}

// exclusive scan, three passes: per-block scan -> scan of block sums -> add
__device__ __forceinline__ int block_exclusive_scan(int v, int *smem, int &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) smem[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (w ? smem[w - 1] : 0);
    total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void k_scan_blocks(const int32_t *in, int32_t *out, int32_t *block_sums, long long m,
                              const int32_t *flags)
{
    if (flags[0] == 0) return;
    __shared__ int sm[32];
    long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
    int v = i < m ? in[i] : 0;
    int total;
    int e = block_exclusive_scan(v, sm, total);
    if (i < m) out[i] = e;
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_top(int32_t *block_sums, int nblocks, int32_t *grand, const int32_t *flags,
                           int *status)
{
    if (flags[0] == 0) return;
    __shared__ int sm[32];
    int carry = 0;
    for (int base = 0; base < nblocks; base += kScanBlock) {
        int i = base + threadIdx.x;
        int v = i < nblocks ? block_sums[i] : 0;
        int total;
        int e = block_exclusive_scan(v, sm, total);
        if (i < nblocks) block_sums[i] = e + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int32_t *out, int32_t *fill, const int32_t *block_sums, long long m,
                           const int32_t *flags)
{
    if (flags[0] == 0) return;
    long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
    if (i < m) {
        int v = out[i] + block_sums[blockIdx.x];
        out[i] = v;
        fill[i] = v;
    }
}

__global__ void k_scatter(const int32_t *atom_bin, int32_t *fill, int32_t *bin_atoms, int n,
                          const int32_t *flags)
{
    if (flags[0] == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int slot = atomicAdd(fill + atom_bin[i], 1);
        bin_atoms[slot] = i;
    }
}

// order each bin's atoms by index so that rows come out deterministic
__global__ void k_sort_bins(const int32_t *bin_start, int32_t *bin_atoms, long long nbins,
                            const int32_t *flags)
{
    if (flags[0] == 0) return;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbins;
         b += (long long)gridDim.x * blockDim.x) {
        int s = bin_start[b], e = bin_start[b + 1];
        for (int k = s + 1; k < e; ++k) {
            int v = bin_atoms[k];
            int q = k - 1;
            while (q >= s && bin_atoms[q] > v) {
                bin_atoms[q + 1] = bin_atoms[q];
                --q;
            }
            bin_atoms[q + 1] = v;
        }
    }
}

// Positions in bin order with the packed image offset (bytes 0-2) and the
// species (byte 3) in .w, so the candidate loop of the row builder reads one
// 16-byte record per candidate instead of chasing bin_atoms -> pos, img,
// species.
__global__ void k_bin_positions(const int32_t *bin_atoms, const float4 *pos, const int32_t *img,
                                const int32_t *species, int n, float4 *pos_bin, const int32_t *flags)
{
    if (flags[0] == 0) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int j = bin_atoms[s];
        float4 p = pos[j];
        p.w = __int_as_float((img[j] & 0xFFFFFF) | (species[j] << 24));
        pos_bin[s] = p;
    }
}

struct RowArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *atom_bin, *img, *bin_start, *bin_atoms;
    const float4 *pos_bin;     // positions in bin order (species in .w)
    int n, max_nbr, compaction;
    const Plan *plans;
    const int32_t *struct_of;
    const float4 *shift;       // [n_structs][kShiftCodes][2] image shifts, FP32 hi and lo
    long long nbins;           // bins of all structures
    int *sched;                // work counter, zero at launch
    float rc2;
    double rc2d;
    int32_t *entries, *count, *group;
    GroupTab *gtab;
    const int32_t *flags;
    int *status;
};

__device__ __forceinline__ int img_comp(int v, int d) { return (int)(int8_t)((v >> (8 * d)) & 0xFF); }

// |r_j + S.cell - r_i|^2 < rc2 decided in FP64 from the exact FP32 inputs
// (used for candidates whose FP32 distance lies close to the cutoff).
__device__ __noinline__ bool within_fp64(const float4 pi, const float4 pj, const int *S, const Plan &P, double rc2)
{
    double tv[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) tv[cc] = S[0] * P.cell[cc] + S[1] * P.cell[3 + cc] + S[2] * P.cell[6 + cc];
    const double x = ((double)pj.x - (double)pi.x) + tv[0];
    const double y = ((double)pj.y - (double)pi.y) + tv[1];
    const double z = ((double)pj.z - (double)pi.z) + tv[2];
    return x * x + y * y + z * z < rc2;
}

// Count, overflow flag and compaction group of a finished row; smask holds
// the species bits of the accepted neighbours, per lane.
__device__ __forceinline__ void finish_row(const RowArgs &a, int i, int cnt, unsigned smask, int lane)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) smask |= __shfl_xor_sync(0xffffffffu, smask, o);
    if (lane == 0) {
        if (cnt > a.max_nbr) {
            // the longest row is only reported with the overflow; one atomic on
            // a single address per atom would serialize every row in one L2 slice
            atomicOr(a.status, kErrOverflow);
            atomicMax(&a.gtab->max_count, cnt);
        }
        a.count[i] = min(cnt, a.max_nbr);
        int g = -1;
        if (cnt > 0) {
            const int si = a.species[i];
            if (si < 0 || si >= kSpecies || (smask >> kSpecies) != 0) atomicOr(a.status, kErrSpecies);
            int cls = 0;
            if (a.compaction) cls = (smask == 1u) ? 1 : (smask == 2u ? 2 : 0);
            g = min(max(si, 0), kSpecies - 1) * 3 + cls;
        }
        a.group[i] = g;
    }
    __syncwarp();
}

// Row of one atom (bin-order index kq), general form: any image of the atoms,
// any stencil, per-atom stencil pruning for orthogonal cells.  The
// candidates of all stencil bins are treated as one sequence (bins in stencil
// order, atoms inside a bin by index), and lanes take 32 consecutive
// candidates at a time, so the lanes stay full however few atoms each bin
// holds.  s_start, s_excl and s_shift are the warp's 32-entry scratch rows.
__device__ __forceinline__ void row_general(const RowArgs &a, int kq, int lane, int *s_start, int *s_excl,
                                            int *s_shift)
{
    const int i = a.bin_atoms[kq];
    const int sidx = structure_of(a.struct_of, i);
    const Plan &P = a.plans[sidx];
    const float4 *img_shift = a.shift + 2 * kShiftCodes * sidx;
    const int span[3] = {2 * P.R[0] + 1, 2 * P.R[1] + 1, 2 * P.R[2] + 1};
    const int n_stencil = span[0] * span[1] * span[2];
    const float4 pib = a.pos_bin[kq];
    const float4 pi = pib;
    const int bin = a.atom_bin[i] - (int)P.bin_base;
    const int bi[3] = {bin / (P.nb[1] * P.nb[2]), (bin / P.nb[2]) % P.nb[1], bin % P.nb[2]};
    const int imi = __float_as_int(pib.w) & 0xFFFFFF;
    // the atom's offset inside its bin (bin units), for skipping stencil
    // bins whose box lies farther than the list cutoff (orthogonal cells)
    float u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float f = pi.x * P.invf[d] + pi.y * P.invf[3 + d] + pi.z * P.invf[6 + d];
        if (P.pbc[d]) f -= floorf(f);
        u[d] = (f - P.flo[d]) / P.fspan[d] * (float)P.nb[d] - (float)bi[d];
    }
    int32_t *row = a.entries + (size_t)i * a.max_nbr;
    int cnt = 0;
    unsigned smask = 0;
    for (int sbase = 0; sbase < n_stencil; sbase += 32) {
        // this lane's stencil bin: range of candidates and lattice shift
        const int k = sbase + lane;
        int c = 0, start = 0, shift = 0;
        if (k < n_stencil) {
            const int dd[3] = {k / (span[1] * span[2]) - P.R[0], (k / span[2]) % span[1] - P.R[1],
                               k % span[2] - P.R[2]};
            int bj[3], sb[3];
            bool skip = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int kk = bi[d] + dd[d];
                if (P.pbc[d]) {
                    const int q = (kk >= 0) ? kk / P.nb[d] : -((-kk + P.nb[d] - 1) / P.nb[d]);
                    sb[d] = q;
                    bj[d] = kk - q * P.nb[d];
                } else {
                    skip |= (kk < 0 || kk >= P.nb[d]);
                    sb[d] = 0;
                    bj[d] = kk;
                }
            }
            if (!skip && P.orth) {
                // lower bound of the distance from the atom to the bin's box
                float d2 = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float gap = dd[d] > 0 ? (float)dd[d] - u[d] : (dd[d] < 0 ? u[d] - (float)dd[d] - 1.f : 0.f);
                    const float gm = fmaxf(gap, 0.f) * P.bw[d];
                    d2 += gm * gm;
                }
                skip = d2 > a.rc2 * 1.0001f + 1e-3f;
            }
            if (!skip) {
                const int b = (int)P.bin_base + (bj[0] * P.nb[1] + bj[1]) * P.nb[2] + bj[2];
                start = a.bin_start[b];
                c = a.bin_start[b + 1] - start;
                shift = (sb[0] & 0xFF) | ((sb[1] & 0xFF) << 8) | ((sb[2] & 0xFF) << 16);
            }
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        s_start[lane] = start;
        s_excl[lane] = incl - c;
        s_shift[lane] = shift;
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int t = base + lane;
            bool ok = false;
            int entry = 0, sj = 0;
            if (t < total) {
                // last stencil slot whose first candidate index is <= t
                int lo = 0, hi = 31;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_excl[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                const int slot = s_start[lo] + (t - s_excl[lo]);
                const int j = a.bin_atoms[slot];
                const float4 pjb = a.pos_bin[slot];   // independent of j: no load chain
                const int sh = s_shift[lo];
                const int imj = __float_as_int(pjb.w) & 0xFFFFFF;
                int S[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) S[d] = img_comp(sh, d) + img_comp(imi, d) - img_comp(imj, d);
                const bool in_range = S[0] >= -2 && S[0] <= 2 && S[1] >= -2 && S[1] <= 2 && S[2] >= -2 &&
                                      S[2] <= 2;
                if (!in_range) atomicOr(a.status, kErrShift);
                const int code = (S[0] + 2) * 25 + (S[1] + 2) * 5 + (S[2] + 2);
                if (in_range && !(j == i && code == kCenterCode)) {
                    const float4 pj = pjb;
                    const float3 r = pair_vector(pi, pj, code, img_shift);
                    const float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
                    if (fabsf(d2 - a.rc2) > 1e-5f * a.rc2) {
                        ok = d2 < a.rc2;
                    } else {
                        // near the cutoff: decide in FP64 from the exact inputs
                        ok = within_fp64(pi, pj, S, P, a.rc2d);
                    }
                    sj = (int)((unsigned)__float_as_int(pjb.w) >> 24);
                    entry = (j << 8) | ((sj & 1) << 7) | code;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            const int slot = cnt + __popc(m & ((1u << lane) - 1u));
            if (ok) {
                if (slot < a.max_nbr) row[slot] = entry;
                smask |= 1u << (sj & 31);
            }
            cnt += __popc(m);
        }
        __syncwarp();
    }
    finish_row(a, i, cnt, smask, lane);
}

constexpr int kBuildWarps = 4;
constexpr int kTile = 320;   // stencil candidates a warp stages for one bin

// One warp per bin (warps claim bins in order from a counter).  For a
// bin whose stencil candidates all carry image 0, image shifts inside
// [-2, 2]^3 and a valid species (always the case for positions wrapped into
// the cell, as in MD), the warp stages the candidate set once: each
// candidate's position relative to the bin's first atom, shifted by its
// image (shifted_diff: within a few 1e-6 A of exact over the stencil's
// extent), and its finished list entry.  Every atom of the bin then scans the
// staged set with one distance test per candidate, decided again in FP64
// from the exact inputs within a relative 4e-5 of the cutoff, so the accepted
// set and its order (stencil order, then atom index) are those of the general
// per-atom path, which the other bins take.
__global__ void __launch_bounds__(kBuildWarps * 32) k_build_bins(RowArgs a)
{
    if (a.flags[0] == 0) return;
    __shared__ int s_start[kBuildWarps][32], s_excl[kBuildWarps][32], s_shift[kBuildWarps][32];
    __shared__ __align__(16) float4 s_cand[kBuildWarps][kTile];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    // one bin per claim: occupied bins cluster in z (the innermost bin
    // index), so a fixed stride would give some warps only empty bins, and
    // bins differ widely in cost
    WarpChunksT<1> wc;
    wc.init(a.sched, (int)a.nbins, lane);
    for (int b = wc.pos(); b < (int)a.nbins; wc.advance(lane), b = wc.pos()) {
        const int k0 = a.bin_start[b], k1 = a.bin_start[b + 1];
        if (k1 <= k0) continue;
        const int sidx = structure_of(a.struct_of, a.bin_atoms[k0]);
        const Plan &P = a.plans[sidx];
        const float4 *img_shift = a.shift + 2 * kShiftCodes * sidx;
        const int span[3] = {2 * P.R[0] + 1, 2 * P.R[1] + 1, 2 * P.R[2] + 1};
        const int n_stencil = span[0] * span[1] * span[2];
        const int bin = b - (int)P.bin_base;
        const int bi[3] = {bin / (P.nb[1] * P.nb[2]), (bin / P.nb[2]) % P.nb[1], bin % P.nb[2]};
        const float4 o4 = a.pos_bin[k0];   // reference point of the staged coordinates
        float4 *cand = s_cand[wl];
        bool fast = true;
        int nc = 0;
        for (int sbase = 0; sbase < n_stencil && fast; sbase += 32) {
            const int k = sbase + lane;
            int c = 0, start = 0, shift = 0;
            if (k < n_stencil) {
                const int dd[3] = {k / (span[1] * span[2]) - P.R[0], (k / span[2]) % span[1] - P.R[1],
                                   k % span[2] - P.R[2]};
                int bj[3], sb[3];
                bool skip = false;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const int kk = bi[d] + dd[d];
                    if (P.pbc[d]) {
                        const int q = (kk >= 0) ? kk / P.nb[d] : -((-kk + P.nb[d] - 1) / P.nb[d]);
                        sb[d] = q;
                        bj[d] = kk - q * P.nb[d];
                    } else {
                        skip |= (kk < 0 || kk >= P.nb[d]);
                        sb[d] = 0;
                        bj[d] = kk;
                    }
                }
                if (!skip) {
                    const int gb = (int)P.bin_base + (bj[0] * P.nb[1] + bj[1]) * P.nb[2] + bj[2];
                    start = a.bin_start[gb];
                    c = a.bin_start[gb + 1] - start;
                    shift = (sb[0] & 0xFF) | ((sb[1] & 0xFF) << 8) | ((sb[2] & 0xFF) << 16);
                }
            }
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            s_start[wl][lane] = start;
            s_excl[wl][lane] = incl - c;
            s_shift[wl][lane] = shift;
            __syncwarp();
            if (nc + total > kTile) {
                fast = false;
            } else {
                for (int base = 0; base < total; base += 32) {
                    const int t = base + lane;
                    bool bad = false;
                    if (t < total) {
                        int lo = 0, hi = 31;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_excl[wl][mid] <= t) lo = mid;
                            else hi = mid - 1;
                        }
                        const int slot = s_start[wl][lo] + (t - s_excl[wl][lo]);
                        const int j = a.bin_atoms[slot];
                        const float4 pj = a.pos_bin[slot];
                        const int sh = s_shift[wl][lo];
                        const int wj = __float_as_int(pj.w);
                        const int sj = (int)((unsigned)wj >> 24);
                        int S[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) S[d] = img_comp(sh, d);
                        bad = (wj & 0xFFFFFF) != 0 || sj >= kSpecies || S[0] < -2 || S[0] > 2 || S[1] < -2 ||
                              S[1] > 2 || S[2] < -2 || S[2] > 2;
                        if (!bad) {
                            const int code = (S[0] + 2) * 25 + (S[1] + 2) * 5 + (S[2] + 2);
                            float3 d;
                            if (code == kCenterCode) {
                                d = make_float3(__fsub_rn(pj.x, o4.x), __fsub_rn(pj.y, o4.y), __fsub_rn(pj.z, o4.z));
                            } else {
                                const float4 th = __ldg(img_shift + 2 * code), tl = __ldg(img_shift + 2 * code + 1);
                                d = make_float3(shifted_diff(pj.x, o4.x, th.x, tl.x), shifted_diff(pj.y, o4.y, th.y, tl.y),
                                                shifted_diff(pj.z, o4.z, th.z, tl.z));
                            }
                            // keep the staged coordinates small, so their rounding stays far below the FP64 band
                            bad = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z))) > 96.f;
                            cand[nc + t] = make_float4(d.x, d.y, d.z, __int_as_float((j << 8) | (sj << 7) | code));
                        }
                    }
                    if (__any_sync(0xffffffffu, bad)) fast = false;
                }
                nc += total;
            }
            __syncwarp();
        }
        if (!fast) {
            for (int kq = k0; kq < k1; ++kq) row_general(a, kq, lane, s_start[wl], s_excl[wl], s_shift[wl]);
            continue;
        }
        for (int kq = k0; kq < k1; ++kq) {
            const int i = a.bin_atoms[kq];
            const float4 pi = a.pos_bin[kq];
            const float dix = __fsub_rn(pi.x, o4.x), diy = __fsub_rn(pi.y, o4.y), diz = __fsub_rn(pi.z, o4.z);
            const int self = (i << 8) | ((int)((unsigned)__float_as_int(pi.w) >> 24) << 7) | kCenterCode;
            int32_t *row = a.entries + (size_t)i * a.max_nbr;
            int cnt = 0;
            unsigned smask = 0;
            for (int base = 0; base < nc; base += 32) {
                const int t = base + lane;
                bool ok = false;
                int e = 0;
                if (t < nc) {
                    const float4 cd = cand[t];
                    e = __float_as_int(cd.w);
                    if (e != self) {
                        const float rx = cd.x - dix, ry = cd.y - diy, rz = cd.z - diz;
                        const float d2 = rx * rx + ry * ry + rz * rz;
                        if (fabsf(d2 - a.rc2) > 4e-5f * a.rc2) {
                            ok = d2 < a.rc2;
                        } else {
                            const int code = e & 127;
                            const int S[3] = {code / 25 - 2, (code / 5) % 5 - 2, code % 5 - 2};
                            ok = within_fp64(pi, __ldg(a.pos + ((unsigned)e >> 8)), S, P, a.rc2d);
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                const int slot = cnt + __popc(m & ((1u << lane) - 1u));
                if (ok) {
                    if (slot < a.max_nbr) row[slot] = e;
                    smask |= 1u << ((e >> 7) & 1);
                }
                cnt += __popc(m);
            }
            finish_row(a, i, cnt, smask, lane);
        }
    }
}

// ---- stable partition of atoms into compaction groups ----
// Each block of 512 atoms packs one 10-bit counter per group into a
// 64-bit word, so one block-wide scan yields every atom's rank in its group.
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v,
                                                             unsigned long long *sm,
                                                             unsigned long long &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        unsigned long long s = lane < nw ? sm[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sm[lane] = s;
    }
    __syncthreads();
    unsigned long long excl = x - v + (w ? sm[w - 1] : 0ull);
    total = sm[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kGroupBlock) k_group_count(const int32_t *group, int n,
                                                             int32_t *blk, const int32_t *flags)
{
    if (flags[0] == 0) return;
    __shared__ unsigned long long sm[32];
    int i = blockIdx.x * kGroupBlock + threadIdx.x;
    int g = i < n ? group[i] : -1;
    unsigned long long v = g >= 0 ? (1ull << (10 * g)) : 0ull;
    unsigned long long total;
    block_scan_u64(v, sm, total);
    if (threadIdx.x < 8)
        blk[blockIdx.x * 8 + threadIdx.x] =
            threadIdx.x < kGroups ? (int)((total >> (10 * threadIdx.x)) & 1023ull) : 0;
}

struct ScanGroupArgs {
    int32_t *blk;
    int nblk;
    int n;
    GroupTab *gtab;
    int ntile_simt[kGroups];
    int nchunk_tc[kGroups];
    const int32_t *flags;
};

__global__ void k_group_scan(ScanGroupArgs a)
{
    if (a.flags[0] == 0) return;
    __shared__ int sm[32];
    __shared__ int totals[kGroups];
    for (int g = 0; g < kGroups; ++g) {
        int carry = 0;
        for (int base = 0; base < a.nblk; base += kScanBlock) {
            int b = base + threadIdx.x;
            int v = b < a.nblk ? a.blk[b * 8 + g] : 0;
            int total;
            int e = block_exclusive_scan(v, sm, total);
            if (b < a.nblk) a.blk[b * 8 + g] = e + carry;
            carry += total;
        }
        if (threadIdx.x == 0) totals[g] = carry;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        GroupTab *t = a.gtab;
        int off_r[2] = {0, 0};
        int assigned = 0;
        for (int g = 0; g < kGroups; ++g) {
            int r = group_region(g);
            t->count[g] = totals[g];
            t->off[g] = off_r[r];
            off_r[r] += totals[g];
            assigned += totals[g];
        }
        t->n_isolated = a.n - assigned;
        t->tiles_simt[0] = 0;
        t->tiles_tc[0] = 0;
        for (int g = 0; g < kGroups; ++g) {
            int mt = (totals[g] + 127) / 128;
            t->tiles_simt[g + 1] = t->tiles_simt[g] + mt * a.ntile_simt[g];
            t->tiles_tc[g + 1] = t->tiles_tc[g] + mt * a.nchunk_tc[g];
        }
    }
}

__global__ void __launch_bounds__(kGroupBlock) k_group_rows(const int32_t *group, int n,
                                                            const int32_t *blk, const GroupTab *gtab,
                                                            int32_t *row, int32_t *atom_of_row,
                                                            int n_cap, const int32_t *flags)
{
    if (flags[0] == 0) return;
    __shared__ unsigned long long sm[32];
    int i = blockIdx.x * kGroupBlock + threadIdx.x;
    int g = i < n ? group[i] : -1;
    unsigned long long v = g >= 0 ? (1ull << (10 * g)) : 0ull;
    unsigned long long total;
    unsigned long long ex = block_scan_u64(v, sm, total);
    if (i < n) {
        if (g >= 0) {
            int rank = (int)((ex >> (10 * g)) & 1023ull);
            int r = gtab->off[g] + blk[blockIdx.x * 8 + g] + rank;
            row[i] = r;
            atom_of_row[group_region(g) * (size_t)n_cap + r] = i;
        } else {
            row[i] = -1;
        }
    }
}

__global__ void k_rebuild_done(int32_t *flags)
{
    if (flags[0]) {
        flags[0] = 0;
        flags[1] += 1;
    }
}

void inverse3(const double *m, double *inv)
{
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                 m[2] * (m[3] * m[7] - m[4] * m[6]);
    inv[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

double width(const double *cell, int d)
{
    const double *a = cell, *b = cell + 3, *c = cell + 6;
    double vol = std::fabs(a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                           a[2] * (b[0] * c[1] - b[1] * c[0]));
    const double *e = cell + 3 * ((d + 1) % 3), *f = cell + 3 * ((d + 2) % 3);
    double x = e[1] * f[2] - e[2] * f[1], y = e[2] * f[0] - e[0] * f[2], z = e[0] * f[1] - e[1] * f[0];
    return vol / std::sqrt(x * x + y * y + z * z);
}

// Cell and inverse of one structure (host); false for a singular cell.
bool plan_cell(Plan &P, const double *cell, const int *pbc)
{
    for (int k = 0; k < 9; ++k) P.cell[k] = cell[k];
    inverse3(cell, P.inv);
    for (int d = 0; d < 3; ++d) P.pbc[d] = pbc[d] ? 1 : 0;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(P.inv[k])) return false;
    for (int k = 0; k < 9; ++k) P.invf[k] = (float)P.inv[k];
    return true;
}

// Bin grid of one structure from its fractional bounding box (host).  Along
// open directions the grid covers the box plus `margin` A on both sides;
// atoms that later leave it are clamped into the edge bins, which stays
// correct because every bin is at least r_c wide.
int plan_grid(Plan &P, const float *bb, double rc, double margin)
{
    long long nbins = 1;
    for (int d = 0; d < 3; ++d) {
        const double w = width(P.cell, d);
        double flo, fspan;
        if (P.pbc[d]) {
            flo = 0.0;
            fspan = 1.0;
        } else {
            double lo = bb[d], hi = bb[3 + d];
            if (!(hi >= lo)) { lo = 0.0; hi = 0.0; }
            flo = lo - margin / w;
            fspan = (hi - lo) + 2.0 * margin / w;
        }
        const double extent = fspan * w;
        int nb = (int)std::floor(extent / (rc * 1.0001));
        nb = std::max(1, std::min(nb, 4096));
        int R = (int)std::ceil(rc / (extent / nb) * (1.0 + 1e-6));
        if (!P.pbc[d]) R = std::min(R, nb);
        if (P.pbc[d] && R > 2 * nb + 1) {
            set_error("neighbour build: periodic cell too narrow for r_cut + skin");
            return FLR_EINVAL;
        }
        P.nb[d] = nb;
        P.R[d] = R;
        P.flo[d] = (float)flo;
        P.fspan[d] = (float)fspan;
        P.bscale[d] = (double)nb / (double)P.fspan[d];
        P.bw[d] = (float)(extent / nb);
        nbins *= nb;
    }
    P.orth = 1;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            if (r != c && P.cell[3 * r + c] != 0.0) P.orth = 0;
    if (nbins > (1ll << 26)) {
        set_error("neighbour build: bin grid too large");
        return FLR_EINVAL;
    }
    P.nbins = nbins;
    return FLR_OK;
}

}  // namespace

// Plan the bin grids of a batch of structures (host, synchronizes once to
// read the bounding boxes) and upload the per-structure tables.
// Fractional bounding box of one structure on the host with the device's
// arithmetic (k_bbox): FP64 products and sums without fused multiply-add
// (this file is compiled with contraction off), rounded to float.
void host_frac_bbox(const double *cell, const float *pos4, int n, float bb[8])
{
    double inv[9];
    inverse3(cell, inv);
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = 0; i < n; ++i) {
        const double x = pos4[4 * (size_t)i], y = pos4[4 * (size_t)i + 1], z = pos4[4 * (size_t)i + 2];
        for (int d = 0; d < 3; ++d) {
            const double a = x * inv[d];
            const double b = y * inv[3 + d];
            const double c = z * inv[6 + d];
            const double s = a + b;
            const float f = (float)(s + c);
            lo[d] = std::min(lo[d], f);
            hi[d] = std::max(hi[d], f);
        }
    }
    for (int d = 0; d < 3; ++d) {
        bb[d] = lo[d];
        bb[3 + d] = hi[d];
    }
    bb[6] = bb[7] = 0.f;
}

// Image shifts S.cell of the 125 codes of one cell (rows = lattice vectors):
// FP64 sums, each split into FP32 hi and lo = RN(t - hi).
void fill_shifts(const double *cl, float4 *out)
{
    for (int code = 0; code < kShiftCodes; ++code) {
        const int S[3] = {code / 25 - 2, (code / 5) % 5 - 2, code % 5 - 2};
        float h[3], l[3];
        for (int d = 0; d < 3; ++d) {
            const double t = S[0] * cl[d] + S[1] * cl[3 + d] + S[2] * cl[6 + d];
            h[d] = (float)t;
            l[d] = (float)(t - (double)h[d]);
        }
        out[2 * code] = make_float4(h[0], h[1], h[2], 0.f);
        out[2 * code + 1] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

// Per-structure tables of a list (offsets, image shifts, plans, bounding
// boxes) for at least n_structs structures; grown by doubling (cudaFree and
// cudaMalloc synchronize the device, so growth is kept rare).
int grow_struct_tables(flr_nbrlist *nl, int n_structs)
{
    if (n_structs <= nl->structs_cap) return FLR_OK;
    cudaFree(nl->offsets_d);
    cudaFree(nl->shift_d);
    cudaFree(nl->plans_d);
    cudaFree(nl->bbox);
    delete[] nl->plans_h;
    delete[] nl->offsets_h;
    const int cap = std::max(n_structs, 2 * nl->structs_cap);
    nl->offsets_d = nullptr;
    nl->shift_d = nullptr;
    nl->plans_d = nullptr;
    nl->bbox = nullptr;
    cudaError_t e = cudaMalloc(&nl->offsets_d, sizeof(int32_t) * (cap + 1));
    if (e == cudaSuccess) e = cudaMalloc(&nl->shift_d, sizeof(float4) * 2 * kShiftCodes * cap);
    if (e == cudaSuccess) e = cudaMalloc(&nl->plans_d, sizeof(Plan) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&nl->bbox, sizeof(float) * 8 * cap);
    nl->plans_h = new Plan[cap];
    nl->offsets_h = new int32_t[cap + 1];
    nl->structs_cap = cap;
    if (e != cudaSuccess) return cuda_fail(e, "batch tables");
    return FLR_OK;
}

// Bin arrays of a list for at least nbins bins (grown by doubling).
int grow_bins(flr_nbrlist *nl, long long nbins)
{
    if (nbins + 1 <= nl->nbins_cap) return FLR_OK;
    cudaFree(nl->bin_start);
    cudaFree(nl->bin_fill);
    nl->bin_start = nullptr;
    nl->bin_fill = nullptr;
    const long long cap = std::max(nbins + 1024, 2 * nl->nbins_cap);
    cudaError_t e = cudaMalloc(&nl->bin_start, sizeof(int32_t) * (cap + 1));
    if (e == cudaSuccess) e = cudaMalloc(&nl->bin_fill, sizeof(int32_t) * (cap + 1));
    if (e != cudaSuccess) return cuda_fail(e, "allocating bins");
    nl->nbins_cap = cap;
    return FLR_OK;
}

int nbrlist_reserve_batch(flr_ctx *ctx, flr_nbrlist *nl, int n_structs, long long nbins)
{
    (void)ctx;
    int s = grow_struct_tables(nl, n_structs);
    if (s == FLR_OK) s = grow_bins(nl, nbins);
    return s;
}

int plan_batch(flr_ctx *ctx, flr_nbrlist *nl, int n_structs, const int32_t *offsets, const double *cells,
               const int32_t *pbc, const float4 *pos, int n, cudaStream_t st, const float *host_bb)
{
    if (n_structs < 1 || offsets[0] != 0 || offsets[n_structs] != n) {
        set_error("neighbour build: batch offsets must start at 0 and end at n_atoms");
        return FLR_EINVAL;
    }
    for (int s = 0; s < n_structs; ++s)
        if (offsets[s + 1] < offsets[s]) {
            set_error("neighbour build: batch offsets must be non-decreasing");
            return FLR_EINVAL;
        }
    {
        const int g = grow_struct_tables(nl, n_structs);
        if (g != FLR_OK) return g;
    }
    nl->n_structs = n_structs;
    for (int s = 0; s <= n_structs; ++s) nl->offsets_h[s] = offsets[s];
    for (int s = 0; s < n_structs; ++s) {
        Plan &P = nl->plans_h[s];
        std::memset(&P, 0, sizeof(Plan));
        if (!plan_cell(P, cells + 9 * s, pbc + 3 * s)) {
            set_error("neighbour build: singular cell matrix (structure " + std::to_string(s) + ")");
            return FLR_EINVAL;
        }
    }
    int r = cuda_fail(cudaMemcpyAsync(nl->plans_d, nl->plans_h, sizeof(Plan) * n_structs, cudaMemcpyHostToDevice, st),
                      "plans");
    if (r == FLR_OK)
        r = cuda_fail(cudaMemcpyAsync(nl->offsets_d, offsets, sizeof(int32_t) * (n_structs + 1), cudaMemcpyHostToDevice,
                                      st),
                      "offsets");
    if (r != FLR_OK) return r;
    // image shifts S.cell of every code: FP64 sums split into FP32 hi + lo
    std::vector<float4> sh(2 * kShiftCodes * (size_t)n_structs);
    for (int s = 0; s < n_structs; ++s) fill_shifts(nl->plans_h[s].cell, sh.data() + 2 * kShiftCodes * (size_t)s);
    r = cuda_fail(cudaMemcpyAsync(nl->shift_d, sh.data(), sizeof(float4) * sh.size(), cudaMemcpyHostToDevice, st),
                  "image shifts");
    if (r != FLR_OK) return r;
    if (n_structs > 1) {
        k_struct_of<<<std::min(n_structs, 65535), 256, 0, st>>>(nl->offsets_d, n_structs, nl->struct_of);
        count_launch(ctx);
    }
    const int32_t *sof = n_structs > 1 ? nl->struct_of : nullptr;
    std::vector<float> bb(8 * (size_t)n_structs, 0.f);
    if (host_bb) {
        std::memcpy(bb.data(), host_bb, sizeof(float) * bb.size());
    } else if (n > 0) {
        const int nb8 = std::max(1, std::min((8 * n_structs + 255) / 256, 1024));
        k_bbox_init<<<nb8, 256, 0, st>>>(reinterpret_cast<int *>(nl->bbox), n_structs);
        const int grid = std::max(1, std::min((n + 255) / 256, ctx->num_sms * 8));
        k_bbox<<<grid, 256, 0, st>>>(pos, n, nl->plans_d, sof, reinterpret_cast<int *>(nl->bbox));
        k_bbox_finish<<<nb8, 256, 0, st>>>(reinterpret_cast<int *>(nl->bbox), n_structs);
        count_launch(ctx, 3);
        r = cuda_fail(cudaMemcpyAsync(bb.data(), nl->bbox, sizeof(float) * bb.size(), cudaMemcpyDeviceToHost, st),
                      "bbox");
        if (r == FLR_OK) r = cuda_fail(cudaStreamSynchronize(st), "bbox");
        if (r != FLR_OK) return r;
    }
    const double rc = ctx->p.r_cut + ctx->p.skin;
    long long base = 0;
    for (int s = 0; s < n_structs; ++s) {
        Plan &P = nl->plans_h[s];
        r = plan_grid(P, bb.data() + 8 * s, rc, 2.0 * rc);
        if (r != FLR_OK) return r;
        P.bin_base = base;
        base += P.nbins;
    }
    if (base > (1ll << 28)) {
        set_error("neighbour build: too many bins in the batch");
        return FLR_EINVAL;
    }
    nl->nbins_total = base;
    {
        const int g = grow_bins(nl, base);
        if (g != FLR_OK) return g;
    }
    nl->plan = nl->plans_h[0];
    nl->planned = true;
    return cuda_fail(cudaMemcpyAsync(nl->plans_d, nl->plans_h, sizeof(Plan) * n_structs, cudaMemcpyHostToDevice, st),
                     "plans");
}

int launch_rebuild(flr_ctx *ctx, flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                   cudaStream_t st, bool wrap_positions, float4 *pos_mut)
{
    const Dims &D = ctx->dims;
    const long long nbins = nl->nbins_total;
    const int nbb = (int)((nbins + kScanBlock - 1) / kScanBlock);
    if (nbb > kScanBlock * 64) {
        set_error("neighbour build: too many bins");
        return FLR_EINVAL;
    }
    const int32_t *sof = nl->n_structs > 1 ? nl->struct_of : nullptr;

    k_zero_bins<<<std::max(1, (int)std::min<long long>((nbins + 255) / 256, 65535)), 256, 0, st>>>(
        nl->bin_fill, nbins, nl->flags);

    BinArgs b;
    b.pos = pos;
    b.pos_mut = wrap_positions ? pos_mut : nullptr;
    b.n = n;
    b.plans = nl->plans_d;
    b.struct_of = sof;
    b.atom_bin = nl->atom_bin;
    b.img = nl->img;
    b.bin_count = nl->bin_fill;
    b.pos_ref = nl->pos_ref;
    b.gtab = nl->gtab;
    b.flags = nl->flags;
    b.status = nl->status;
    k_bin<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 8)), 256, 0, st>>>(b);

    // bin_start = exclusive scan of counts; block sums live in blk_group's tail
    int32_t *bsums = nl->blk_group + (size_t)8 * ((nl->n_cap + kGroupBlock - 1) / kGroupBlock + 1);
    k_scan_blocks<<<nbb, kScanBlock, 0, st>>>(nl->bin_fill, nl->bin_start, bsums, nbins, nl->flags);
    k_scan_top<<<1, kScanBlock, 0, st>>>(bsums, nbb, nl->bin_start + nbins, nl->flags, nl->status);
    k_scan_add<<<nbb, kScanBlock, 0, st>>>(nl->bin_start, nl->bin_fill, bsums, nbins, nl->flags);
    k_scatter<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 8)), 256, 0, st>>>(nl->atom_bin, nl->bin_fill,
                                                                                        nl->bin_atoms, n, nl->flags);
    k_sort_bins<<<(int)std::max<long long>(1, std::min<long long>((nbins + 255) / 256, ctx->num_sms * 8)), 256, 0,
                  st>>>(nl->bin_start, nl->bin_atoms, nbins, nl->flags);
    k_bin_positions<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 8)), 256, 0, st>>>(
        nl->bin_atoms, wrap_positions ? pos_mut : pos, nl->img, species, n, nl->pos_bin, nl->flags);

    RowArgs r;
    r.pos = wrap_positions ? pos_mut : pos;
    r.species = species;
    r.atom_bin = nl->atom_bin;
    r.img = nl->img;
    r.bin_start = nl->bin_start;
    r.bin_atoms = nl->bin_atoms;
    r.pos_bin = nl->pos_bin;
    r.n = n;
    r.max_nbr = nl->max_nbr;
    r.compaction = ctx->p.compaction;
    r.plans = nl->plans_d;
    r.shift = nl->shift_d;
    r.struct_of = sof;
    const double rc = ctx->p.r_cut + ctx->p.skin;
    r.rc2 = (float)(rc * rc);
    r.rc2d = rc * rc;
    r.entries = nl->entries;
    r.count = nl->count;
    r.group = nl->group;
    r.gtab = nl->gtab;
    r.flags = nl->flags;
    r.status = nl->status;
    r.nbins = nbins;
    r.sched = nl->sched;
    {
        const cudaError_t e = cudaMemsetAsync(r.sched, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "list build work counter");
    }
    k_build_bins<<<persistent_grid(k_build_bins, kBuildWarps * 32, ctx->num_sms, (nbins + kBuildWarps - 1) / kBuildWarps),
                   kBuildWarps * 32, 0, st>>>(r);

    const int nblk = (n + kGroupBlock - 1) / kGroupBlock;
    k_group_count<<<nblk, kGroupBlock, 0, st>>>(nl->group, n, nl->blk_group, nl->flags);
    ScanGroupArgs sg;
    sg.blk = nl->blk_group;
    sg.nblk = nblk;
    sg.n = n;
    sg.gtab = nl->gtab;
    for (int g = 0; g < kGroups; ++g) {
        const int reg = group_region(g);
        sg.ntile_simt[g] = (2 * D.K[reg] + 143) / 144;
        sg.nchunk_tc[g] = 1;   // the tensor-core kernel walks the column chunks of an M-tile itself
    }
    sg.flags = nl->flags;
    k_group_scan<<<1, kScanBlock, 0, st>>>(sg);
    k_group_rows<<<nblk, kGroupBlock, 0, st>>>(nl->group, n, nl->blk_group, nl->gtab, nl->row,
                                               nl->atom_of_row, nl->n_cap, nl->flags);
    k_rebuild_done<<<1, 1, 0, st>>>(nl->flags);
    count_launch(ctx, FLR_REBUILD_KERNELS);
    return cuda_fail(cudaGetLastError(), "neighbour rebuild");
}

namespace {

__global__ void k_rebuild_cond(cudaGraphConditionalHandle h, const int32_t *flags)
{
    cudaGraphSetConditional(h, flags[0] != 0 ? 1u : 0u);
}

// Every host-side value the rebuild sequence bakes into its launches.
constexpr int kKeyWords = 40;
struct RebuildGraph {
    cudaGraphExec_t exec;
    unsigned long long key[kKeyWords];
};

void rebuild_key(const flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 bool wrap, const float4 *pos_mut, unsigned long long *k)
{
    int q = 0;
    auto put = [&](unsigned long long v) { k[q++] = v; };
    auto ptr = [&](const void *v) { put(reinterpret_cast<uintptr_t>(v)); };
    ptr(pos); ptr(species); put((unsigned long long)n); put(wrap ? 1 : 0); ptr(pos_mut);
    put((unsigned long long)nl->nbins_total); put((unsigned long long)nl->n_structs); ptr(nl->struct_of);
    ptr(nl->bin_fill); ptr(nl->bin_start); ptr(nl->bin_atoms); ptr(nl->atom_bin); ptr(nl->img);
    ptr(nl->pos_ref); ptr(nl->pos_bin); ptr(nl->gtab); ptr(nl->flags); ptr(nl->status); ptr(nl->sched);
    ptr(nl->plans_d); ptr(nl->shift_d); ptr(nl->blk_group); put((unsigned long long)nl->n_cap);
    put((unsigned long long)nl->max_nbr); ptr(nl->entries); ptr(nl->count); ptr(nl->group); ptr(nl->row);
    ptr(nl->atom_of_row);
    put((unsigned long long)ctx->num_sms); put((unsigned long long)ctx->p.compaction);
    double rc = ctx->p.r_cut, sk = ctx->p.skin;
    unsigned long long b;
    std::memcpy(&b, &rc, 8); put(b);
    std::memcpy(&b, &sk, 8); put(b);
    put((unsigned long long)ctx->dims.K[0]); put((unsigned long long)ctx->dims.K[1]);
    while (q < kKeyWords) put(0);
}

}  // namespace

void free_rebuild_graph(flr_nbrlist *nl)
{
    RebuildGraph *rg = reinterpret_cast<RebuildGraph *>(nl->rgraph);
    if (!rg) return;
    if (rg->exec) cudaGraphExecDestroy(rg->exec);
    delete rg;
    nl->rgraph = nullptr;
}

int launch_rebuild_cond(flr_ctx *ctx, flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                        cudaStream_t st, bool wrap_positions, float4 *pos_mut)
{
    unsigned long long key[kKeyWords];
    rebuild_key(ctx, nl, pos, species, n, wrap_positions, pos_mut, key);
    RebuildGraph *rg = reinterpret_cast<RebuildGraph *>(nl->rgraph);
    if (!rg || std::memcmp(rg->key, key, sizeof(key)) != 0) {
        free_rebuild_graph(nl);
        // graph: [k_rebuild_cond] -> [if (flag) { the rebuild sequence }]
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaGraphCreate(&g, 0);
        cudaGraphConditionalHandle h = 0;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
        cudaGraphNode_t n_cond = nullptr, n_if = nullptr;
        if (e == cudaSuccess) {
            cudaKernelNodeParams kp = {};
            const int32_t *flags = nl->flags;
            void *args[] = {&h, &flags};
            kp.func = reinterpret_cast<void *>(k_rebuild_cond);
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&n_cond, g, nullptr, 0, &kp);
        }
        cudaGraphNodeParams cp = {};
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&n_if, g, &n_cond, nullptr, 1, &cp);
        }
        int s = FLR_OK;
        if (e == cudaSuccess) {
            // record the sequence into the body on a private stream (no work runs)
            cudaStream_t cs = nullptr;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e == cudaSuccess) {
                e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const long long launches = ctx->launches;
                    s = launch_rebuild(ctx, nl, pos, species, n, cs, wrap_positions, pos_mut);
                    ctx->launches = launches;   // counted per graph launch instead
                    cudaGraph_t body = nullptr;
                    const cudaError_t e2 = cudaStreamEndCapture(cs, &body);
                    if (e == cudaSuccess) e = e2;
                }
                cudaStreamDestroy(cs);
            }
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && s == FLR_OK) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (s != FLR_OK) return s;
        if (e != cudaSuccess) return cuda_fail(e, "conditional rebuild graph");
        rg = new RebuildGraph();
        rg->exec = exec;
        std::memcpy(rg->key, key, sizeof(key));
        nl->rgraph = rg;
    }
    // one kernel per step; the sequence's 14 kernels only on rebuild steps
    count_launch(ctx, 1);
    return cuda_fail(cudaGraphLaunch(rg->exec, st), "conditional rebuild graph launch");
}

}  // namespace flr

// ---------------------------------------------------------------------------
// Neighbour build that allocates nothing (flr_build_neighbors_noalloc).
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// fixed at start-up (a serving process that reserves its whole budget once,
// or a host framework that owns every device allocation through its own
// pool) and callers that hold no library context.  This entry point runs the
// same cell-list kernels as flr_build_neighbors, but every buffer besides the
// caller's inputs and outputs (bin counts and starts, the per-atom bin and
// image tables, the bin-sorted atom order, scan block sums, the grid plan,
// the status word) lives in one file-scope device array of fixed size,
// kNoAllocBytes (about 3.9 MB), that each GPU loading this library keeps
// until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace flr {
namespace {

constexpr int kNoAllocMaxAtoms = 1 << 16;
constexpr int kNoAllocMaxBins = 1 << 16;
constexpr size_t kNoAllocBytes =
    (size_t)kNoAllocMaxAtoms * (5 * sizeof(int32_t) + 2 * sizeof(float4)) +   // bin, img, sorted atoms, group, spare;
                                                                            // pos_ref, positions in bin order
    (size_t)2 * (kNoAllocMaxBins + 2) * sizeof(int32_t) +                  // bin starts, bin fill
    (size_t)(kNoAllocMaxBins / kScanBlock + 2) * sizeof(int32_t) +         // scan block sums
    (size_t)2 * kShiftCodes * sizeof(float4) + 256 +                        // image shifts
    4096;                                                                   // flags, status, bbox, plan, group table

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256];   // device address of g_noalloc_scratch, per device ordinal

}  // namespace
}  // namespace flr

// The scratch itself.  Host code must not use this name as a pointer (on the
// host it is only a stand-in symbol); the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[flr::kNoAllocBytes];

extern "C" int flr_build_neighbors_noalloc(const flr_system *sys, double r_list, int32_t max_nbr, int32_t *entries,
                                           int32_t *count, flr_stream_t stream)
{
    using namespace flr;
    if (!sys || sys->n_atoms < 0 || !(r_list > 0.0) || max_nbr < 32 || max_nbr > 512 || max_nbr % 32) {
        set_error("flr_build_neighbors_noalloc: invalid argument (r_list > 0, max_nbr a multiple of 32 in [32, 512])");
        return FLR_EINVAL;
    }
    const int n = sys->n_atoms;
    if (n > kNoAllocMaxAtoms) {
        set_error("flr_build_neighbors_noalloc: " + std::to_string(n) + " atoms exceed the fixed scratch limit of " +
                  std::to_string(kNoAllocMaxAtoms) + "; use flr_build_neighbors");
        return FLR_EINVAL;
    }
    if (n > 0 && (!sys->pos || !sys->species || !entries || !count)) {
        set_error("flr_build_neighbors_noalloc: null pointer");
        return FLR_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(sys->pos) % 16) {
        set_error("flr_build_neighbors_noalloc: pos must be 16-byte aligned float[n][4]");
        return FLR_EINVAL;
    }
    if (n == 0) return FLR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    int s = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != FLR_OK) return s;
    if (dev < 0 || dev >= 256) {
        set_error("flr_build_neighbors_noalloc: device ordinal out of range");
        return FLR_EINVAL;
    }
    // once per device, with that device current: the device address of the scratch array
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }
    int num_sms = 1;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);

    // carve the scratch
    unsigned char *q = static_cast<unsigned char *>(base);
    auto take = [&q](size_t bytes) {
        unsigned char *p = q;
        q += (bytes + 255) & ~size_t(255);
        return p;
    };
    int32_t *atom_bin = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * kNoAllocMaxAtoms));
    int32_t *img = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * kNoAllocMaxAtoms));
    int32_t *bin_atoms = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * kNoAllocMaxAtoms));
    int32_t *group = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * kNoAllocMaxAtoms));
    float4 *pos_ref = reinterpret_cast<float4 *>(take(sizeof(float4) * kNoAllocMaxAtoms));
    float4 *pos_bin = reinterpret_cast<float4 *>(take(sizeof(float4) * kNoAllocMaxAtoms));
    int32_t *bin_start = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (kNoAllocMaxBins + 2)));
    int32_t *bin_fill = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (kNoAllocMaxBins + 2)));
    int32_t *bsums = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (kNoAllocMaxBins / kScanBlock + 2)));
    int32_t *flags = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * 4));
    int *status = reinterpret_cast<int *>(take(sizeof(int) * 4));
    float *bbox = reinterpret_cast<float *>(take(sizeof(float) * 8));
    Plan *plan_d = reinterpret_cast<Plan *>(take(sizeof(Plan)));
    GroupTab *gtab = reinterpret_cast<GroupTab *>(take(sizeof(GroupTab)));
    float4 *shift_d = reinterpret_cast<float4 *>(take(sizeof(float4) * 2 * kShiftCodes));
    int *sched = reinterpret_cast<int *>(take(sizeof(int)));
    if (q > static_cast<unsigned char *>(base) + kNoAllocBytes) {
        set_error("flr_build_neighbors_noalloc: scratch layout exceeds the array");
        return FLR_EINVAL;
    }

    // bin grid from the fractional bounding box (host reads six floats)
    Plan P;
    std::memset(&P, 0, sizeof(P));
    if (!plan_cell(P, sys->cell, sys->pbc)) {
        set_error("flr_build_neighbors_noalloc: singular cell");
        return FLR_EINVAL;
    }
    s = cuda_fail(cudaMemcpyAsync(plan_d, &P, sizeof(Plan), cudaMemcpyHostToDevice, st), "plan");
    if (s != FLR_OK) return s;
    float4 sh[2 * kShiftCodes];
    fill_shifts(P.cell, sh);
    s = cuda_fail(cudaMemcpyAsync(shift_d, sh, sizeof(sh), cudaMemcpyHostToDevice, st), "image shifts");
    if (s != FLR_OK) return s;
    const float4 *pos = reinterpret_cast<const float4 *>(sys->pos);
    k_bbox_init<<<1, 32, 0, st>>>(reinterpret_cast<int *>(bbox), 1);
    k_bbox<<<std::max(1, std::min((n + 255) / 256, num_sms * 8)), 256, 0, st>>>(pos, n, plan_d, nullptr,
                                                                              reinterpret_cast<int *>(bbox));
    k_bbox_finish<<<1, 32, 0, st>>>(reinterpret_cast<int *>(bbox), 1);
    float bb[8];
    s = cuda_fail(cudaMemcpyAsync(bb, bbox, sizeof(bb), cudaMemcpyDeviceToHost, st), "bbox");
    if (s == FLR_OK) s = cuda_fail(cudaStreamSynchronize(st), "bbox");
    if (s != FLR_OK) return s;
    s = plan_grid(P, bb, r_list, 2.0 * r_list);
    if (s != FLR_OK) return s;
    const long long nbins = P.nbins;
    if (nbins > kNoAllocMaxBins) {
        set_error("flr_build_neighbors_noalloc: the bin grid needs " + std::to_string(nbins) +
                  " bins, above the fixed scratch limit of " + std::to_string(kNoAllocMaxBins));
        return FLR_EINVAL;
    }
    P.bin_base = 0;
    // the array keeps the previous call's contents: reset what must start at zero
    s = cuda_fail(cudaMemcpyAsync(plan_d, &P, sizeof(Plan), cudaMemcpyHostToDevice, st), "plan");
    if (s == FLR_OK) s = cuda_fail(cudaMemsetAsync(status, 0, sizeof(int) * 4, st), "reset scratch");
    if (s == FLR_OK) s = cuda_fail(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, st), "reset scratch");
    if (s == FLR_OK) s = cuda_fail(cudaMemsetAsync(flags, 1, 1, st), "reset scratch");   // rebuild flag on
    if (s != FLR_OK) return s;

    k_zero_bins<<<std::max(1, (int)std::min<long long>((nbins + 255) / 256, 65535)), 256, 0, st>>>(bin_fill, nbins,
                                                                                                   flags);
    BinArgs b;
    b.pos = pos;
    b.pos_mut = nullptr;
    b.n = n;
    b.plans = plan_d;
    b.struct_of = nullptr;
    b.atom_bin = atom_bin;
    b.img = img;
    b.bin_count = bin_fill;
    b.pos_ref = pos_ref;
    b.gtab = gtab;
    b.flags = flags;
    b.status = status;
    k_bin<<<std::max(1, std::min((n + 255) / 256, num_sms * 8)), 256, 0, st>>>(b);
    const int nbb = (int)((nbins + kScanBlock - 1) / kScanBlock);
    k_scan_blocks<<<nbb, kScanBlock, 0, st>>>(bin_fill, bin_start, bsums, nbins, flags);
    k_scan_top<<<1, kScanBlock, 0, st>>>(bsums, nbb, bin_start + nbins, flags, status);
    k_scan_add<<<nbb, kScanBlock, 0, st>>>(bin_start, bin_fill, bsums, nbins, flags);
    k_scatter<<<std::max(1, std::min((n + 255) / 256, num_sms * 8)), 256, 0, st>>>(atom_bin, bin_fill, bin_atoms, n,
                                                                                  flags);
    k_sort_bins<<<(int)std::max<long long>(1, std::min<long long>((nbins + 255) / 256, num_sms * 8)), 256, 0, st>>>(
        bin_start, bin_atoms, nbins, flags);
    k_bin_positions<<<std::max(1, std::min((n + 255) / 256, num_sms * 8)), 256, 0, st>>>(bin_atoms, pos, img,
                                                                                        sys->species, n, pos_bin, flags);
    RowArgs r;
    r.pos = pos;
    r.species = sys->species;
    r.atom_bin = atom_bin;
    r.img = img;
    r.bin_start = bin_start;
    r.bin_atoms = bin_atoms;
    r.pos_bin = pos_bin;
    r.n = n;
    r.max_nbr = max_nbr;
    r.compaction = 1;
    r.plans = plan_d;
    r.shift = shift_d;
    r.struct_of = nullptr;
    r.rc2 = (float)(r_list * r_list);
    r.rc2d = r_list * r_list;
    r.entries = entries;
    r.count = count;
    r.group = group;
    r.gtab = gtab;
    r.flags = flags;
    r.status = status;
    r.nbins = nbins;
    r.sched = sched;
    s = cuda_fail(cudaMemsetAsync(sched, 0, sizeof(int), st), "list build work counter");
    if (s != FLR_OK) return s;
    k_build_bins<<<persistent_grid(k_build_bins, kBuildWarps * 32, num_sms, (nbins + kBuildWarps - 1) / kBuildWarps),
                   kBuildWarps * 32, 0, st>>>(r);
    s = cuda_fail(cudaGetLastError(), "neighbour build (no allocation)");
    if (s != FLR_OK) return s;
    int stv = 0, maxc = 0;
    s = cuda_fail(cudaMemcpyAsync(&stv, status, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    if (s == FLR_OK)
        s = cuda_fail(cudaMemcpyAsync(&maxc, &gtab->max_count, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    if (s == FLR_OK) s = cuda_fail(cudaStreamSynchronize(st), "neighbour build (no allocation)");
    if (s != FLR_OK) return s;
    if (stv & kErrOverflow) {
        set_error("neighbour list overflow: an atom has " + std::to_string(maxc) + " neighbours, max_nbr is " +
                  std::to_string(max_nbr));
        return FLR_ENBR_OVERFLOW;
    }
    if (stv & kErrShift) {
        set_error("image shift out of range (positions far outside the cell, or cell too narrow)");
        return FLR_EDEVICE;
    }
    if (stv & kErrSpecies) {
        set_error("species index out of range");
        return FLR_EINVAL;
    }
    return FLR_OK;
}
