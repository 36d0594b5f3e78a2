// Gather-tiled x phase of the B300 HPR-LP solver (sm_103a): the normal iterations' A^T y
// of eq. (update-x) with the gathered vector y staged in shared memory.
//
// The sliced-ELL phase kernel (k_sell) gathers one random 8-byte entry of y from L2 per
// stored entry of A^T, and B300 serves such gathers at ~0.95 per clock per SM: on the
// medium planted LP (5.25 M gathers a phase) that rate is one of the x phase's three
// ceilings, beside HBM and FP64 issue.  Shared memory serves random 8-byte loads ~5x
// faster.  So y is cut into blocks of
// consecutive entries that fit one CTA's shared memory, and A^T into the sub-matrices
// T_b holding the entries whose column (a row of A) lies in block b:
//
//   k_tile_part: CTA c stages block b = cta_blk[c] of y in shared memory and its warps
//                take work units of T_b from block b's counter (sliced ELL as in k_sell,
//                column offsets within the block in 16 bits); each sub-row's sum (the
//                part of one row of A^T y that block b holds) is stored in its own slot of
//                the partial-sum buffer P.
//   k_tile_epi:  row j of A^T adds its slots slot_ptr[j] .. slot_ptr[j+1]-1 in block order
//                and applies the x update of the FP64 form (EpiX<false>::row, unchanged).
//
// Every sub-row's sum is a fixed function of the layout and the slots are added in a fixed
// order, so results are bitwise reproducible whichever CTA takes which unit.  The row sums
// are those of the sliced-ELL kernel in another order of addition (FP64 throughout).
//
// Measured on the medium planted LP, the pair is slower than k_sell (41 against 35 us):
// the split adds FP64 instructions (a row becomes up to one sub-row per block, each with
// its own chain merge; one add per slot; the epilogue in a kernel of its own), and FP64
// issue is B300's scarcest resource.  The layout is therefore opt-in
// (hpr_options.gather_tiles).
#pragma once

#include "hpr_device.cuh"

namespace hprdev {

#ifndef HPR_TILE_TB
#define HPR_TILE_TB 1024
#endif
#ifndef HPR_TILE_BATCH
#define HPR_TILE_BATCH 8
#endif
constexpr int TILE_TB = HPR_TILE_TB;         // threads of a k_tile_part CTA (one CTA per SM)
constexpr int TILE_BATCH = HPR_TILE_BATCH;   // steps whose loads a warp issues together
constexpr int TILE_MAX_BLOCKS = TB;          // k_tile_epi's first CTA resets the counters

struct TileArgs {
    const int *cta_blk;          // block of each CTA
    const int *bstart;           // nblk + 1: first entry of the gathered vector in each block
    const int *ustart;           // nblk + 1: first work unit of each block
    const int *wstart;           // units + 1: first slice of each unit (a run of slices)
    const int4 *smeta;           // slices: first sub-row, first stored entry, steps (32
                                 // entries each), log2 lanes per sub-row | sub-rows << 8
    const int *oslot;            // sub-rows: slot of the sub-row's sum in P
    const double *val;           // stored values (padding: 0)
    const unsigned short *col;   // column offset within the block (padding: 0)
    double *P;                   // partial sums, one slot per (row, block) pair
    unsigned *ctr;               // per block: work units taken (k_tile_epi resets them)
    const double *g;             // the gathered vector (y)
    int trigger_from;            // programmatic launch: CTAs from this index on let the next
                                 // kernel start once they have waited for the previous one
};

struct TileEpiArgs {
    int rows, nblk;
    const int *slot_ptr;         // rows + 1
    const double *P;
    unsigned *ctr;
    int trigger_from;
};

// One slice: lanes accumulate their sub-row's entries (two FMA chains over the batches of
// TILE_BATCH steps, the last 1 .. TILE_BATCH-1 steps on the first chain), the lanes of a
// sub-row are added by a fixed xor butterfly and the sub-row's first lane stores the sum.
__device__ __forceinline__ void tile_slice(const TileArgs &A, const double *gs, int glen, int4 meta, int lane)
{
    const int r0 = meta.x, base = meta.y, steps = meta.z;
    const int lg = meta.w & 0xff, nrows = meta.w >> 8;
    const int q = lane >> lg;                    // sub-row q of the slice: lanes q L .. q L + L - 1
    const bool owner = (lane & ((1 << lg) - 1)) == 0 && q < nrows;
    const int slot = owner ? A.oslot[r0 + q] : 0;
    const double *pv = A.val + base + lane;
    const unsigned short *pc = A.col + base + lane;
    double a0 = 0.0, a1 = 0.0;
    int k = 0;
    for (; k + TILE_BATCH <= steps; k += TILE_BATCH) {
        double v[TILE_BATCH];
        int c[TILE_BATCH];
#pragma unroll
        for (int u = 0; u < TILE_BATCH; ++u) {
            v[u] = __ldcs(pv + (k + u) * 32);
            c[u] = HPR_COL((int)__ldcs(pc + (k + u) * 32), glen);
        }
#pragma unroll
        for (int u = 0; u < TILE_BATCH; u += 2) {
            a0 = fma(v[u], gs[c[u]], a0);
            a1 = fma(v[u + 1], gs[c[u + 1]], a1);
        }
    }
    const bool two = k > 0;                      // warp-uniform: the second chain was used
    if (k < steps) {
        const int rem = steps - k;               // warp-uniform, 1 .. TILE_BATCH-1
        double v[TILE_BATCH - 1];
        int c[TILE_BATCH - 1];
#pragma unroll
        for (int u = 0; u < TILE_BATCH - 1; ++u) {   // the loads together (predicated)
            v[u] = u < rem ? __ldcs(pv + (k + u) * 32) : 0.0;
            c[u] = u < rem ? HPR_COL((int)__ldcs(pc + (k + u) * 32), glen) : 0;
        }
#pragma unroll
        for (int u = 0; u < TILE_BATCH - 1; ++u) {   // only the FMAs of real steps
            if (u >= rem) break;
            a0 = fma(v[u], gs[c[u]], a0);
        }
    }
    if (two) a0 += a1;
    for (int o = 1; o < (1 << lg); o <<= 1) a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    if (owner) A.P[slot] = a0;
}

__global__ void __launch_bounds__(TILE_TB, 1) k_tile_part(TileArgs A)
{
    extern __shared__ __align__(16) double gs[];
    const int b = A.cta_blk[blockIdx.x];
    const int g0 = A.bstart[b], glen = A.bstart[b + 1] - g0;   // g0 is even
    const int u0 = A.ustart[b], nu = A.ustart[b + 1] - u0;
    const int lane = threadIdx.x & 31;
    asm volatile("griddepcontrol.wait;" ::: "memory");        // y is the previous kernel's output
    if ((int)blockIdx.x >= A.trigger_from) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // each warp takes its first unit now and its next one a unit ahead, so that the counter's
    // round trip overlaps the work
    unsigned mine = lane == 0 ? atomicAdd(A.ctr + b, 1u) : 0u;
    {   // the block of y into shared memory: 16-byte asynchronous copies, all in flight at once
        const double2 *src = reinterpret_cast<const double2 *>(A.g + g0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(gs);
        for (int i = threadIdx.x; i < (glen >> 1); i += TILE_TB)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * (unsigned)i), "l"(src + i)
                         : "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        if ((glen & 1) && threadIdx.x == 0) gs[glen - 1] = __ldcg(A.g + g0 + glen - 1);
    }
    __syncthreads();
    unsigned cur = __shfl_sync(0xffffffffu, mine, 0);
    while (cur < (unsigned)nu) {
        mine = lane == 0 ? atomicAdd(A.ctr + b, 1u) : 0u;
        const int U = u0 + (int)cur;
        const int s_end = A.wstart[U + 1];
        int s = A.wstart[U];
        int4 meta = A.smeta[s];
        for (; s < s_end; ++s) {
            const int4 next = s + 1 < s_end ? A.smeta[s + 1] : meta;   // a slice ahead
            tile_slice(A, gs, glen, meta, lane);
            meta = next;
        }
        cur = __shfl_sync(0xffffffffu, mine, 0);
    }
}

// the x update of a normal iteration from the partial sums: one thread per row of A^T, the
// row's slots added in block order (four loads in flight at a time)
template <class E>
__global__ void __launch_bounds__(TB) k_tile_epi(TileEpiArgs T, E e)
{
    static_assert(E::NP == 0, "normal iterations only");
    e.load();
    const int j = blockIdx.x * TB + threadIdx.x;
    const bool act = j < T.rows;
    typename E::Pre pre{};
    int q0 = 0, q1 = 0;
    if (act) {
        pre = e.prefetch(j);                     // neither written by k_tile_part
        q0 = T.slot_ptr[j];
        q1 = T.slot_ptr[j + 1];
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if ((int)blockIdx.x >= T.trigger_from) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (blockIdx.x == 0 && (int)threadIdx.x < T.nblk) T.ctr[threadIdx.x] = 0u;   // k_tile_part has ended
    if (!act) return;
    double s = 0.0;
    int q = q0;
    if (q < q1) s = T.P[q++];
    for (; q + 4 <= q1; q += 4) {
        const double p0 = T.P[q], p1 = T.P[q + 1], p2 = T.P[q + 2], p3 = T.P[q + 3];
        s += p0;
        s += p1;
        s += p2;
        s += p3;
    }
    if (q < q1) {
        const int rem = q1 - q;                  // 1 .. 3
        const double p0 = T.P[q], p1 = rem > 1 ? T.P[q + 1] : 0.0, p2 = rem > 2 ? T.P[q + 2] : 0.0;
        s += p0;
        if (rem > 1) s += p1;
        if (rem > 2) s += p2;
    }
    const double sums[2] = {s, s};
    double part[1] = {0.0};
    e.row(j, true, sums, pre, part);
}

}  // namespace hprdev
