// mg_query.cu -- segment histograms of boxes: footprint assembly (Sec. 3.6,
// Algorithm 1) and the reverse weight push through the Mixture Graph.
//
// Plan (one warp per box): clip the box, split each axis range into aligned
// power-of-two runs (footprint_1d), count the blocks of the runs' tensor
// product and the cubes tiling them (a block of run levels (lx, ly, lz) sits at
// level l = min and holds 2^(lx-l) * 2^(ly-l) * 2^(lz-l) cubes), then write one
// 12-byte record per block: first cube index, the index of its first cube in
// the level's ID array, level, and log2 extents.  Blocks follow Algorithm 1's
// loop order (z, y, x).  Every level is stored three times (x-, y- and
// z-fastest); a block reads the copy whose fastest axis is its longest side,
// so even a one-voxel-thick slab reads contiguous IDs.
//
// Main (persistent CTAs, MG_SCHED_BATCHED): a global ticket hands out chunks of
// `chunk` consecutive cubes of one box; each warp of the CTA takes a
// contiguous span of the chunk.  While 32 or more cubes of the current block
// remain, the warp walks the block directly (one ID per lane, 32-bit index
// arithmetic); the last few cubes of a block go with the next block's first
// ones through a ballot that tells each lane its block.  Adjacent lanes with
// the same (level, node) merge into one contribution of count * 8^l.  A
// source adds it to the CTA's shared-memory histogram; an internal node is
// queued per warp and pushed down its lerp tree 32 at a time (p gets
// W*a/(a+b), q gets W*b/(a+b), exact u32 arithmetic) into the same histogram.
// At the end of a chunk the touched bins are added to the box's row in global
// memory -- the only global atomics.
//
// MG_SCHED_PLAIN is the baseline: one launch and one CTA per box, walking the
// blocks in order.
#include "mg_internal.cuh"

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

namespace mg {
namespace {

constexpr int kMaxRuns = 40;
constexpr int kMaxStack = 64;
constexpr uint32_t kMaxSharedSegments = 32768;
constexpr uint32_t kMaxPushSteps = 1u << 24;   // a valid table never needs this many

struct Geom {
    int L;
    int id0_bytes;
    uint32_t S;
    int32_t dims[MG_MAX_LEVELS][3];
    // offset of level l >= 1 in copy c's concatenated levels
    int64_t off[MG_MAX_LEVELS][3];
    // strides of the second and third axis of each copy (copy 0: x, y, z;
    // copy 1: y, z, x; copy 2: z, x, y): the row pitch and pitch x middle dim
    uint32_t st1[MG_MAX_LEVELS][3], st2[MG_MAX_LEVELS][3];
    // bit l of vec_ok[c] / vec32_ok[c]: every row of copy c at level l starts
    // on a 16-byte / 32-byte boundary (row pitch and level offset multiples)
    uint32_t vec_ok[3], vec32_ok[3];
};

struct Ids {
    const void* l0[3];       // level 0 copies (uint16 or uint32)
    const uint32_t* hi[3];   // levels >= 1 copies, concatenated at Geom::off
};

struct Blk {
    uint32_t start;   // first cube of the block within its box
    uint32_t base;    // index of the block's first cube in its copy of level l
    uint32_t meta;    // l | copy << 5 | e0 << 7 | e1 << 12 | e2 << 17 (log2 extents, copy axis order)
};

Geom make_geom(const mg_graph* g) {
    Geom G;
    G.L = g->L;
    G.id0_bytes = g->id0_bytes;
    G.S = g->S;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        for (int k = 0; k < 3; k++) G.dims[l][k] = g->geom.dims[l][k];
        const uint32_t dx = (uint32_t)G.dims[l][0], dy = (uint32_t)G.dims[l][1], dz = (uint32_t)G.dims[l][2];
        const uint32_t mid[3] = {dy, dz, dx};
        for (int c = 0; c < 3; c++) {
            G.off[l][c] = g->qoff[l][c];
            const uint32_t pitch = l < g->L ? (uint32_t)g->qpitch[l][c] : 1u;
            G.st1[l][c] = pitch;
            G.st2[l][c] = pitch * mid[c];
        }
    }
    for (int c = 0; c < 3; c++) {
        G.vec_ok[c] = G.vec32_ok[c] = 0;
        for (int l = 0; l < G.L && l < MG_MAX_LEVELS; l++) {
            const uint32_t per16 = l == 0 ? 16u / (uint32_t)G.id0_bytes : 4u;   // IDs per 16 bytes
            const bool ok = G.st1[l][c] % per16 == 0 && G.st2[l][c] % per16 == 0 &&
                            (l == 0 || G.off[l][c] % per16 == 0);
            const uint32_t per32 = 2 * per16;
            const bool ok32 = G.st1[l][c] % per32 == 0 && G.st2[l][c] % per32 == 0 &&
                              (l == 0 || G.off[l][c] % per32 == 0);
            if (ok) G.vec_ok[c] |= 1u << l;
            if (ok32) G.vec32_ok[c] |= 1u << l;
        }
    }
    return G;
}

Ids make_ids(const mg_graph* g) {
    Ids I;
    for (int c = 0; c < 3; c++) {
        I.l0[c] = g->mip0x[c].p ? g->mip0x[c].p : g->mip0.p;   // copy 0 may be mip0 itself
        I.hi[c] = g->mipx[c].as<uint32_t>();
    }
    return I;
}

// block of run levels (lx, ly, lz) whose origin is the level-0 voxel (x0, y0, z0)
__device__ __forceinline__ Blk make_blk(const Geom& G, uint32_t start, int32_t x0, int32_t y0, int32_t z0, int lx,
                                        int ly, int lz) {
    const int l = min(lx, min(ly, lz));
    const int ex = lx - l, ey = ly - l, ez = lz - l;
    const uint32_t X = (uint32_t)x0 >> l, Y = (uint32_t)y0 >> l, Z = (uint32_t)z0 >> l;
    int c, e0, e1, e2;
    uint32_t base;
    if (ex >= ey && ex >= ez) {
        c = 0; e0 = ex; e1 = ey; e2 = ez;
        base = Z * G.st2[l][0] + Y * G.st1[l][0] + X;
    } else if (ey >= ez) {
        c = 1; e0 = ey; e1 = ez; e2 = ex;
        base = X * G.st2[l][1] + Z * G.st1[l][1] + Y;
    } else {
        c = 2; e0 = ez; e1 = ex; e2 = ey;
        base = Y * G.st2[l][2] + X * G.st1[l][2] + Z;
    }
    Blk B;
    B.start = start;
    B.base = base;
    B.meta = (uint32_t)(l | c << 5 | e0 << 7 | e1 << 12 | e2 << 17);
    return B;
}

// Algorithm 1, footprint_1d: aligned power-of-two steps covering [i, i+di)
// clipped to [0, dim); tzcnt(0) is infinite.
__device__ __forceinline__ int footprint_1d(int64_t i, int64_t di, int64_t dim, uint8_t* r, int32_t* start) {
    int n = 0;
    di = min(i + di, dim) - i;
    while (di > 0 && n < kMaxRuns) {
        const int a = 63 - __clzll(di);
        const int b = i == 0 ? 63 : __ffsll(i) - 1;
        const int l = min(a, b);
        r[n] = (uint8_t)l;
        start[n] = (int32_t)i;
        n++;
        di -= (int64_t)1 << l;
        i += (int64_t)1 << l;
    }
    return n;
}

__device__ __forceinline__ bool box_ok(const int32_t* b, const Geom& G) {
    return b[0] >= 0 && b[0] < G.dims[0][0] && b[1] >= 0 && b[1] < G.dims[0][1] && b[2] >= 0 &&
           b[2] < G.dims[0][2] && b[3] >= 1 && b[4] >= 1 && b[5] >= 1;
}

struct Runs {
    uint8_t lx[kMaxRuns], ly[kMaxRuns], lz[kMaxRuns];
    int32_t sx[kMaxRuns], sy[kMaxRuns], sz[kMaxRuns];
    int nx, ny, nz;
};

__device__ __forceinline__ void make_runs(const int32_t* b, const Geom& G, Runs& R) {
    R.nx = footprint_1d(b[0], b[3], G.dims[0][0], R.lx, R.sx);
    R.ny = footprint_1d(b[1], b[4], G.dims[0][1], R.ly, R.sy);
    R.nz = footprint_1d(b[2], b[5], G.dims[0][2], R.lz, R.sz);
}

// the runs of a warp's box, one axis per lane, into the warp's shared slot
__device__ __forceinline__ void make_runs_warp(const int32_t* b, const Geom& G, Runs& R) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) R.nx = footprint_1d(b[0], b[3], G.dims[0][0], R.lx, R.sx);
    else if (lane == 1) R.ny = footprint_1d(b[1], b[4], G.dims[0][1], R.ly, R.sy);
    else if (lane == 2) R.nz = footprint_1d(b[2], b[5], G.dims[0][2], R.lz, R.sz);
    __syncwarp();
}

constexpr int kPlanThreads = 256;   // plan kernels: one warp per box

__device__ __forceinline__ uint32_t block_cubes(int lx, int ly, int lz) {
    const int l = min(lx, min(ly, lz));
    return 1u << (lx + ly + lz - 3 * l);
}

// Footprint cubes of a box in closed form.  On each axis let F(m) be the sum
// over its runs of level a >= m of 2^(a-m), and P(m) = Fx(m) Fy(m) Fz(m).  A
// block of run levels (a, b, c) with minimum m0 adds 2^(a+b+c-3m) to P(m) for
// every m <= m0, so the blocks' cubes, sum 2^(a+b+c-3 m0), equal
// P(0) - 7 * sum over m >= 1 of P(m).  Algorithm 1's steps on one axis rise
// to a peak and fall again, so no level occurs more than twice and two bit
// masks hold an axis's levels: F(m) = (once >> m) + (twice >> m).
__device__ __forceinline__ void level_masks(const uint8_t* l, int n, uint64_t& once, uint64_t& twice) {
    once = twice = 0;
    for (int i = 0; i < n; i++) {
        const uint64_t bit = 1ull << l[i];
        if (once & bit) twice |= bit;
        else once |= bit;
    }
}

__device__ __forceinline__ uint64_t cubes_from_masks(uint64_t x1, uint64_t x2, uint64_t y1, uint64_t y2, uint64_t z1,
                                                     uint64_t z2) {
    const uint64_t p0 = (x1 + x2) * (y1 + y2) * (z1 + z2);
    uint64_t rest = 0;
    for (int m = 1; m < 64 && (x1 >> m) && (y1 >> m) && (z1 >> m); m++)
        rest += ((x1 >> m) + (x2 >> m)) * ((y1 >> m) + (y2 >> m)) * ((z1 >> m) + (z2 >> m));
    return p0 - 7 * rest;
}

__device__ __forceinline__ uint64_t footprint_cubes(const Runs& R) {
    uint64_t x1, x2, y1, y2, z1, z2;
    level_masks(R.lx, R.nx, x1, x2);
    level_masks(R.ly, R.ny, y1, y2);
    level_masks(R.lz, R.nz, z1, z2);
    return cubes_from_masks(x1, x2, y1, y2, z1, z2);
}

// Batch size and capacities read on the device, for query plans replayed as
// CUDA graphs: the launches cover Q boxes, *Qd of them are live, and the
// footprint must fit the plan's buffers.  Qd == nullptr: all Q are live and
// the buffers were sized for this batch.
struct Lim {
    const int64_t* Qd;
    uint64_t cap_blocks, cap_chunks;
};

__device__ __forceinline__ int64_t live_q(const Lim& lim, int64_t Q) { return lim.Qd ? *lim.Qd : Q; }

__device__ __forceinline__ bool over_cap(const Lim& lim, const uint64_t* blk_off, const uint64_t* chunk_off,
                                         int64_t Qe) {
    return lim.Qd && (blk_off[Qe] > lim.cap_blocks || chunk_off[Qe] > lim.cap_chunks);
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
__global__ void plan_count_kernel(Geom G, const int32_t* __restrict__ boxes, int64_t Q, uint32_t chunk,
                                  uint32_t* __restrict__ nblk, uint64_t* __restrict__ ncube,
                                  uint64_t* __restrict__ nchunk, unsigned* __restrict__ status, Lim lim) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= Q) return;
    if (q >= live_q(lim, Q)) {
        if (lane == 0) {
            if (nblk) nblk[q] = 0;
            ncube[q] = 0;
            if (nchunk) nchunk[q] = 0;
        }
        return;
    }
    int32_t b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
    if (!box_ok(b, G)) {
        if (lane == 0) {
            set_status(status, kStatBadInput);
            if (nblk) nblk[q] = 0;
            ncube[q] = 0;
            if (nchunk) nchunk[q] = 0;
        }
        return;
    }
    __shared__ Runs wr[kPlanThreads / 32];
    Runs& R = wr[threadIdx.x >> 5];
    make_runs_warp(b, G, R);
    if (lane == 0) {
        const uint64_t cubes = footprint_cubes(R);
        if (nblk) nblk[q] = (uint32_t)(R.nx * R.ny * R.nz);
        ncube[q] = cubes;
        if (nchunk) nchunk[q] = (cubes + chunk - 1) / chunk;
    }
}

// Block records of every box, and for every work chunk of `chunk` cubes its
// box and the block holding its first cube.
__global__ void plan_write_kernel(Geom G, const int32_t* __restrict__ boxes, int64_t Q,
                                  const uint64_t* __restrict__ blk_off, Blk* __restrict__ blk, Lim lim,
                                  const uint64_t* __restrict__ chunk_off, uint32_t chunk,
                                  uint32_t* __restrict__ chunk_q, uint32_t* __restrict__ chunk_b) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t Qe = live_q(lim, Q);
    if (q >= Qe || over_cap(lim, blk_off, chunk_off, Qe)) return;
    int32_t b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
    if (!box_ok(b, G)) return;
    __shared__ Runs wr[kPlanThreads / 32];
    Runs& R = wr[threadIdx.x >> 5];
    make_runs_warp(b, G, R);
    const uint64_t base = blk_off[q], cbase = chunk_off[q];
    const int npairs = R.ny * R.nz;
    uint32_t running = 0;
    for (int pbase = 0; pbase < npairs; pbase += 32) {
        const int pr = pbase + lane;
        const bool valid = pr < npairs;
        const int j = valid ? pr % R.ny : 0, k = valid ? pr / R.ny : 0;
        uint32_t row = 0;
        if (valid)
            for (int i = 0; i < R.nx; i++) row += block_cubes(R.lx[i], R.ly[j], R.lz[k]);
        // exclusive warp scan of the row totals
        uint32_t incl = row;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (valid) {
            uint32_t start = running + incl - row;
            for (int i = 0; i < R.nx; i++) {
                const uint64_t bi = base + (uint64_t)pr * R.nx + i;
                const uint32_t n = block_cubes(R.lx[i], R.ly[j], R.lz[k]);
                blk[bi] = make_blk(G, start, R.sx[i], R.sy[j], R.sz[k], R.lx[i], R.ly[j], R.lz[k]);
                // the chunks whose first cube lies in this block
                for (uint64_t c = ((uint64_t)start + chunk - 1) / chunk; c * chunk < (uint64_t)start + n; c++) {
                    chunk_q[cbase + c] = (uint32_t)q;
                    chunk_b[cbase + c] = (uint32_t)bi;
                }
                start += n;
            }
        }
        running += tot;
    }
}

// ---------------------------------------------------------------------------
// The plan of a query-plan run in one launch: the footprint counts of every
// box, both exclusive scans in a single pass, the zeroing of the batch's
// output rows, the block records and the chunk map.  CTAs take tiles of `tb`
// boxes in ticket order (tb chosen on the host so that the tiles of a full
// batch fill the GPU once); a tile publishes its own totals, then sums its
// predecessors' words backwards until it meets one that holds an inclusive
// prefix, and publishes its own prefix.  Plans only (capacities in `lim`).
// ---------------------------------------------------------------------------
constexpr int kTileMax = 64;                     // boxes per tile at most
constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kBoxLanes = 8;                     // lanes per box in the count phase (three build runs)
constexpr int kBoxGroups = kFusedThreads / kBoxLanes;
constexpr int kScanPerLane = kTileMax / 32;      // boxes per lane in the tile scan
constexpr int kFusedItems = 6;                   // blocks per thread and round, interleaved
constexpr int kLookWindows = 4;                  // look-back windows of 32 tiles loaded per poll
constexpr uint64_t kTileAgg = 1ull << 62;        // the word holds the tile's own total
constexpr uint64_t kTilePre = 2ull << 62;        // the word holds the inclusive prefix
constexpr uint64_t kTileVal = (1ull << 62) - 1;
constexpr unsigned kLookbackLimit = 1u << 20;    // polls before the look-back gives up

// boxes per tile for a batch of Q: about one tile per resident CTA
int tile_boxes(int64_t Q, int sms) {
    const int64_t slots = (int64_t)sms * 2;
    return (int)std::min<int64_t>(kTileMax, std::max<int64_t>(1, (Q + slots - 1) / slots));
}

// zero the tile words of the live batch and both work tickets
__global__ void plan_reset_kernel(const int64_t* __restrict__ Qd, int tb, uint64_t* __restrict__ tiles,
                                  unsigned long long* __restrict__ tickets) {
    const int64_t n = 2 * ((*Qd + tb - 1) / tb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        tiles[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 2) tickets[threadIdx.x] = 0;
}

struct FusedOut {
    uint64_t* ncube;
    uint64_t* blk_off;
    uint64_t* chunk_off;
    Blk* blk;
    uint32_t* chunk_q;
    uint32_t* chunk_b;
    uint64_t* tiles;               // two words per tile: blocks, chunks
    unsigned long long* ticket;    // tile order
    uint32_t* acc;                 // rows zeroed for the live batch
    float* accf;                   // likewise (fp32 histograms), or nullptr
    void* const* io;               // io[0]: the boxes; io[1]: the output (acc for u32, accf for fp32)
};

// Algorithm 1's steps on one axis (as footprint_1d) together with the axis's
// level masks (levels seen once, levels seen twice)
__device__ __forceinline__ int axis_runs(int64_t i, int64_t di, int64_t dim, uint8_t* r, int32_t* start,
                                         uint64_t& once, uint64_t& twice) {
    int n = 0;
    once = twice = 0;
    di = min(i + di, dim) - i;
    while (di > 0 && n < kMaxRuns) {
        const int a = 63 - __clzll(di);
        const int b = i == 0 ? 63 : __ffsll(i) - 1;
        const int l = min(a, b);
        const uint64_t bit = 1ull << l;
        if (once & bit) twice |= bit;
        else once |= bit;
        r[n] = (uint8_t)l;
        start[n] = (int32_t)i;
        n++;
        di -= (int64_t)1 << l;
        i += (int64_t)1 << l;
    }
    return n;
}

// zero a[r0, r1) of 4-byte elements (a 4-byte aligned) with 16-byte stores
// between the unaligned ends
template <typename T>
__device__ __forceinline__ void zero_span(T* a, size_t r0, size_t r1) {
    static_assert(sizeof(T) == 4, "4-byte elements");
    const size_t lead = ((16u - (reinterpret_cast<uintptr_t>(a + r0) & 15u)) & 15u) / 4u;
    const size_t a0 = min(r0 + lead, r1), a1 = a0 + ((r1 - a0) & ~(size_t)3);
    for (size_t i = r0 + threadIdx.x; i < a0; i += kFusedThreads) a[i] = T(0);
    for (size_t i = a1 + threadIdx.x; i < r1; i += kFusedThreads) a[i] = T(0);
    uint4* v = reinterpret_cast<uint4*>(a + a0);
    for (size_t i = threadIdx.x; i < (a1 - a0) / 4; i += kFusedThreads) v[i] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(kFusedThreads, 2) plan_fused_kernel(Geom G, const int32_t* __restrict__ boxes,
                                                                      int64_t Q, int tb, uint32_t chunk,
                                                                      int chunk_shift, Lim lim, FusedOut F,
                                                                      unsigned* __restrict__ status) {
    __shared__ Runs wr[kTileMax];
    __shared__ uint32_t s_nblk[kTileMax];
    __shared__ uint64_t s_ncube[kTileMax];
    __shared__ uint64_t s_mx[kTileMax], s_my[kTileMax];   // ceil(2^32 / nx), ceil(2^32 / ny)
    __shared__ uint32_t s_boff[kTileMax + 1];   // tile-local block offsets, total last
    __shared__ uint64_t s_coff[kTileMax + 1];   // tile-local chunk offsets, total last
    __shared__ uint32_t s_cube[kTileMax];       // tile-local cube offsets, mod 2^32
    __shared__ uint32_t s_wsum[kFusedWarps][kFusedItems];
    __shared__ uint32_t s_rtot[kFusedItems];
    __shared__ unsigned long long s_tile;
    __shared__ uint64_t s_pre_b, s_pre_c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(F.ticket, 1ull);
    // the main kernel may be scheduled once every tile has started; it waits
    // for this grid's completion before it reads anything written here
    grid_dependents_launch();
    __syncthreads();
    const int64_t tile = (int64_t)s_tile;
    const int64_t Qe = live_q(lim, Q);
    const int64_t q0 = tile * tb;
    if (q0 >= Qe) return;   // no tile of the live batch waits on this one
    uint32_t* acc = F.acc;
    float* accf = F.accf;
    if (F.io) {
        boxes = static_cast<const int32_t*>(F.io[0]);
        if (accf) accf = static_cast<float*>(F.io[1]);
        else acc = static_cast<uint32_t*>(F.io[1]);
    }

    // 1. blocks and cubes of every box: kBoxLanes lanes per box, lanes 0-2 of
    // a group building one axis's runs each
    const int grp = threadIdx.x / kBoxLanes, bl = threadIdx.x % kBoxLanes;
    for (int w0 = 0; w0 < tb; w0 += kBoxGroups) {
        const int w = w0 + grp;
        const int64_t q = q0 + w;
        const bool live = w < tb && q < Qe;
        bool ok = false;
        uint64_t once = 0, twice = 0;
        if (live) {
            int32_t b[6];
#pragma unroll
            for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
            ok = box_ok(b, G);
            if (!ok && bl == 0) set_status(status, kStatBadInput);
            if (ok && bl < 3) {
                Runs& R = wr[w];
                const int64_t i0 = bl == 0 ? b[0] : bl == 1 ? b[1] : b[2];
                const int64_t di = bl == 0 ? b[3] : bl == 1 ? b[4] : b[5];
                const int64_t dim = bl == 0 ? G.dims[0][0] : bl == 1 ? G.dims[0][1] : G.dims[0][2];
                uint8_t* lv = bl == 0 ? R.lx : bl == 1 ? R.ly : R.lz;
                int32_t* sv = bl == 0 ? R.sx : bl == 1 ? R.sy : R.sz;
                const int n = axis_runs(i0, di, dim, lv, sv, once, twice);
                if (bl == 0) R.nx = n;
                else if (bl == 1) R.ny = n;
                else R.nz = n;
            }
        }
        // lanes 1 and 2 of a group hand their masks to lane 0
        const uint64_t y1 = __shfl_down_sync(0xffffffffu, once, 1, kBoxLanes);
        const uint64_t y2 = __shfl_down_sync(0xffffffffu, twice, 1, kBoxLanes);
        const uint64_t z1 = __shfl_down_sync(0xffffffffu, once, 2, kBoxLanes);
        const uint64_t z2 = __shfl_down_sync(0xffffffffu, twice, 2, kBoxLanes);
        __syncwarp();
        if (bl == 0 && w < tb) {
            uint64_t cubes = 0;
            uint32_t nb = 0;
            if (ok) {
                const Runs& R = wr[w];
                cubes = cubes_from_masks(once, twice, y1, y2, z1, z2);
                nb = (uint32_t)(R.nx * R.ny * R.nz);
                s_mx[w] = ((1ull << 32) + R.nx - 1) / (uint64_t)R.nx;
                s_my[w] = ((1ull << 32) + R.ny - 1) / (uint64_t)R.ny;
            }
            if (live) F.ncube[q] = cubes;
            s_nblk[w] = nb;
            s_ncube[w] = cubes;
        }
    }
    {   // the tile's live output rows are one contiguous span
        const size_t r0 = (size_t)q0 * G.S, r1 = (size_t)min(q0 + tb, Qe) * G.S;
        zero_span(acc, r0, r1);
        if (accf) zero_span(accf, r0, r1);
    }
    __syncthreads();

    // 2. offsets within the tile (kScanPerLane consecutive boxes per lane),
    // then the prefix of all earlier tiles
    if (warp == 0) {
        uint64_t nbk[kScanPerLane], nck[kScanPerLane], nqk[kScanPerLane];
        uint64_t xb = 0, xc = 0, xq = 0;
#pragma unroll
        for (int k = 0; k < kScanPerLane; k++) {
            const int w = lane * kScanPerLane + k;
            nbk[k] = w < tb ? s_nblk[w] : 0u;
            nqk[k] = w < tb ? s_ncube[w] : 0u;
            nck[k] = chunk_shift >= 0 ? (nqk[k] + chunk - 1) >> chunk_shift : (nqk[k] + chunk - 1) / chunk;
            xb += nbk[k];
            xc += nck[k];
            xq += nqk[k];
        }
        uint64_t ib = xb, ic = xc, iq = xq;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t yb = __shfl_up_sync(0xffffffffu, ib, o);
            const uint64_t yc = __shfl_up_sync(0xffffffffu, ic, o);
            const uint64_t yq = __shfl_up_sync(0xffffffffu, iq, o);
            if (lane >= o) {
                ib += yb;
                ic += yc;
                iq += yq;
            }
        }
        uint64_t ob = ib - xb, oc = ic - xc, oq = iq - xq;
#pragma unroll
        for (int k = 0; k < kScanPerLane; k++) {
            s_boff[lane * kScanPerLane + k] = (uint32_t)ob;
            s_coff[lane * kScanPerLane + k] = oc;
            s_cube[lane * kScanPerLane + k] = (uint32_t)oq;
            ob += nbk[k];
            oc += nck[k];
            oq += nqk[k];
        }
        const uint64_t agg_b = __shfl_sync(0xffffffffu, ib, 31), agg_c = __shfl_sync(0xffffffffu, ic, 31);
        if (lane == 0) {
            s_boff[kTileMax] = (uint32_t)agg_b;
            s_coff[kTileMax] = agg_c;
        }
        uint64_t* word = F.tiles + 2 * tile;
        if (lane == 0) {
            const uint64_t flag = tile == 0 ? kTilePre : kTileAgg;
            st_relaxed_u64(word, flag | agg_b);
            st_relaxed_u64(word + 1, flag | agg_c);
        }
        // look back kLookWindows windows of 32 tiles per poll; a word pair
        // counts once both words carry the same flag
        uint64_t eb = 0, ec = 0;
        int64_t top = tile - 1;
        unsigned polls = 0;
        bool done = top < 0;
        while (!done) {
            uint64_t wb[kLookWindows], wc[kLookWindows];
#pragma unroll
            for (int k = 0; k < kLookWindows; k++) {
                const int64_t t = top - lane - 32 * k;
                wb[k] = wc[k] = kTilePre;   // before the first tile: prefix 0
                if (t >= 0) {
                    wb[k] = ld_relaxed_u64(F.tiles + 2 * t);
                    wc[k] = ld_relaxed_u64(F.tiles + 2 * t + 1);
                }
            }
            bool late_seen = false;
#pragma unroll
            for (int k = 0; k < kLookWindows; k++) {
                if (done || late_seen) continue;
                const bool ready = (wb[k] >> 62) != 0 && (wb[k] >> 62) == (wc[k] >> 62);
                const unsigned pre = __ballot_sync(0xffffffffu, ready && (wb[k] >> 62) == 2u);
                const unsigned late = __ballot_sync(0xffffffffu, !ready);
                // the lanes up to the nearest tile holding its prefix are needed
                const unsigned need = pre ? ((pre & (0u - pre)) << 1) - 1u : 0xffffffffu;
                if (late & need) {
                    late_seen = true;
                    continue;
                }
                const bool use = (need >> lane) & 1u;
                uint64_t vb = use ? wb[k] & kTileVal : 0u, vc = use ? wc[k] & kTileVal : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vb += __shfl_xor_sync(0xffffffffu, vb, o);
                    vc += __shfl_xor_sync(0xffffffffu, vc, o);
                }
                eb += vb;
                ec += vc;
                if (pre) done = true;
                else top -= 32;
            }
            if (late_seen && !done) {
                if (++polls > kLookbackLimit) {
                    if (lane == 0) set_status(status, kStatTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        if (lane == 0) {
            if (tile > 0) {
                st_relaxed_u64(word, kTilePre | (eb + agg_b));
                st_relaxed_u64(word + 1, kTilePre | (ec + agg_c));
            }
            s_pre_b = eb;
            s_pre_c = ec;
        }
    }
    __syncthreads();
    const uint64_t pre_b = s_pre_b, pre_c = s_pre_c;
    const uint64_t tot_b = pre_b + s_boff[kTileMax], tot_c = pre_c + s_coff[kTileMax];
    for (int w = threadIdx.x; w < tb; w += kFusedThreads) {
        const int64_t q = q0 + w;
        if (q >= Qe) break;
        F.blk_off[q] = pre_b + s_boff[w];
        F.chunk_off[q] = pre_c + s_coff[w];
        if (q == Qe - 1) {
            F.blk_off[Qe] = tot_b;
            F.chunk_off[Qe] = tot_c;
            if (tot_b > lim.cap_blocks || tot_c > lim.cap_chunks) set_status(status, kStatCapacity);
        }
    }
    // past the plan's buffers: the last tile has flagged the batch, nothing is written
    if (tot_b > lim.cap_blocks || tot_c > lim.cap_chunks) return;

    // 3. block records and the chunk map; item `it` of thread t is the tile's
    // block r0 + it * kFusedThreads + t.  A box's block t is row pr = t / nx,
    // column i = t - pr nx; the quotients by nx, ny < 2^16 of numerators
    // < 2^16 are exact as (n * ceil(2^32 / d)) >> 32.
    const uint32_t nbt = s_boff[kTileMax];
    uint32_t carry = 0;   // cubes of the earlier rounds, mod 2^32
    for (uint32_t r0 = 0; r0 < nbt; r0 += kFusedThreads * kFusedItems) {
        uint32_t n[kFusedItems], incl[kFusedItems];
        int wk[kFusedItems], ik[kFusedItems], jk[kFusedItems], kk[kFusedItems];
#pragma unroll
        for (int it = 0; it < kFusedItems; it++) {
            const uint32_t idx = r0 + it * kFusedThreads + threadIdx.x;
            n[it] = 0;
            wk[it] = ik[it] = jk[it] = kk[it] = 0;
            if (idx < nbt) {
                int w = 0;   // the last box whose blocks start at or before idx
#pragma unroll
                for (int st = kTileMax / 2; st > 0; st >>= 1)
                    if (s_boff[w + st] <= idx) w += st;
                const Runs& R = wr[w];
                const uint32_t t = idx - s_boff[w];
                const uint32_t pr = (uint32_t)(((uint64_t)t * s_mx[w]) >> 32);
                const uint32_t k = (uint32_t)(((uint64_t)pr * s_my[w]) >> 32);
                wk[it] = w;
                ik[it] = (int)(t - pr * (uint32_t)R.nx);
                jk[it] = (int)(pr - k * (uint32_t)R.ny);
                kk[it] = (int)k;
                n[it] = block_cubes(R.lx[ik[it]], R.ly[jk[it]], R.lz[kk[it]]);
            }
            uint32_t v = n[it];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            incl[it] = v;
            if (lane == 31) s_wsum[warp][it] = v;
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int it = 0; it < kFusedItems; it++) {
                const uint32_t x = lane < kFusedWarps ? s_wsum[lane][it] : 0u;
                uint32_t v = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += y;
                }
                __syncwarp();
                if (lane < kFusedWarps) s_wsum[lane][it] = v - x;
                if (lane == 31) s_rtot[it] = v;
            }
        }
        __syncthreads();
        uint32_t base = carry;
#pragma unroll
        for (int it = 0; it < kFusedItems; it++) {
            const uint32_t idx = r0 + it * kFusedThreads + threadIdx.x;
            if (idx < nbt) {
                const int w = wk[it], i = ik[it], j = jk[it], k = kk[it];
                const Runs& R = wr[w];
                const uint32_t start = base + s_wsum[warp][it] + incl[it] - n[it] - s_cube[w];
                const uint64_t bi = pre_b + idx;
                F.blk[bi] = make_blk(G, start, R.sx[i], R.sy[j], R.sz[k], R.lx[i], R.ly[j], R.lz[k]);
                const uint64_t cb = pre_c + s_coff[w];
                const uint64_t first = (uint64_t)start + chunk - 1;
                for (uint64_t c = chunk_shift >= 0 ? first >> chunk_shift : first / chunk;
                     c * chunk < (uint64_t)start + n[it]; c++) {
                    F.chunk_q[cb + c] = (uint32_t)(q0 + w);
                    F.chunk_b[cb + c] = (uint32_t)bi;
                }
            }
            base += s_rtot[it];
        }
        carry = base;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// shared-memory histogram of one chunk
// ---------------------------------------------------------------------------
template <bool FP>
struct Hist {
    uint32_t* h;        // S integer bins
    float* hf;          // S fractional bins (fp32 push)
    uint16_t* touched;  // bins to flush (when tracking)
    uint32_t* ntouched;
    bool track;         // false: the flush scans all S bins, adds need no return value

    __device__ __forceinline__ void add_int(uint32_t s, uint32_t w) const {
        if (track) {
            if (atomicAdd(h + s, w) == 0u) touched[atomicAdd(ntouched, 1u)] = (uint16_t)s;
        } else {
            atomicAdd(h + s, w);
        }
    }
    __device__ __forceinline__ void add_frac(uint32_t s, float w) const {
        if (track) {
            if (atomicAdd(hf + s, w) == 0.f) touched[atomicAdd(ntouched, 1u)] = (uint16_t)s;
        } else {
            atomicAdd(hf + s, w);
        }
    }
};

// segment counts up to this are flushed by scanning every bin
constexpr uint32_t kScanFlushMax = 2048;
// segment counts up to this get one histogram per warp
constexpr uint32_t kWarpHistMax = 2048;

template <typename AT> struct AlphaCvt;
template <> struct AlphaCvt<float> {
    static __device__ __forceinline__ float to(float x) { return x; }
};
template <> struct AlphaCvt<__half> {
    static __device__ __forceinline__ float to(__half x) { return __half2float(x); }
};
template <> struct AlphaCvt<__nv_bfloat16> {
    static __device__ __forceinline__ float to(__nv_bfloat16 x) { return __bfloat162float(x); }
};

struct PushArgs {
    const uint2* pq;
    const uint2* ab32;
    const void* alpha;
    uint32_t S;
    unsigned* status;
    const uint2* lut_meta;   // mixture lookup table (null: walk the lerp trees)
    const uint2* lut;
};

// The table row of node n for a push of weight w: entries (source, count)
// scaled to 8^lmin, so each source receives (w >> 3 lmin) * count.  len = 0
// when n has no row or w is not a multiple of 8^lmin (then the tree is walked).
__device__ __forceinline__ void lut_row(const PushArgs& P, uint32_t n, uint32_t w, uint32_t& off, uint32_t& len,
                                        uint32_t& k) {
    const uint2 m = __ldg(P.lut_meta + n);
    const uint32_t lm = 3u * (m.y & 255u);
    len = m.y >> 8;
    off = m.x;
    k = w >> lm;
    if (len && (k << lm) != w) len = 0;
}

// exact integer push of weight W from node n (Sec. 3.6 with the lerp tree of
// Sec. 3.2): depth-first, one branch kept in registers, the other stacked
template <bool FP>
__device__ void push_int(const PushArgs& P, const Hist<FP>& H, uint32_t n, uint32_t w) {
    uint32_t sn[kMaxStack], sw[kMaxStack];
    int sp = 0;
    for (uint32_t step = 0;; step++) {
        if (step >= kMaxPushSteps) {
            set_status(P.status, kStatInexact);
            return;
        }
        if (n < P.S) {
            H.add_int(n, w);
            if (sp == 0) return;
            --sp;
            n = sn[sp];
            w = sw[sp];
            continue;
        }
        const uint2 e = __ldg(P.pq + n);
        const uint2 ab = __ldg(P.ab32 + n);
        const uint32_t s = ab.x + ab.y;
        const uint32_t k = s ? w / s : 0u;
        if (s == 0 || k * s != w || sp >= kMaxStack) {
            set_status(P.status, kStatInexact);
            if (sp == 0) return;
            --sp;
            n = sn[sp];
            w = sw[sp];
            continue;
        }
        sn[sp] = e.y;
        sw[sp] = k * ab.y;
        sp++;
        n = e.x;
        w = k * ab.x;
    }
}

// fp32 push: q receives W*alpha, p the rest
template <typename AT>
__device__ void push_frac(const PushArgs& P, const Hist<true>& H, uint32_t n, float w) {
    uint32_t sn[kMaxStack];
    float sw[kMaxStack];
    int sp = 0;
    const AT* alpha = static_cast<const AT*>(P.alpha);
    for (uint32_t step = 0;; step++) {
        if (step >= kMaxPushSteps) {
            set_status(P.status, kStatInexact);
            return;
        }
        if (n < P.S) {
            H.add_frac(n, w);
            if (sp == 0) return;
            --sp;
            n = sn[sp];
            w = sw[sp];
            continue;
        }
        const uint2 e = __ldg(P.pq + n);
        float al = AlphaCvt<AT>::to(alpha[n]);
        uint32_t p = e.x, q = e.y;
        if (al < 0.f) {   // 16-bit weights: sign = p and q swapped, |alpha| <= 1/2
            al = -al;
            p = e.y;
            q = e.x;
        }
        if (sp >= kMaxStack) {
            set_status(P.status, kStatInexact);
            return;
        }
        const float wq = w * al;
        sn[sp] = q;
        sw[sp] = wq;
        sp++;
        n = p;
        w = w - wq;
    }
}

// the push of one (node, weight) by one lane: its mixture-table row, else its
// lerp tree
template <bool FP, typename AT>
__device__ __noinline__ void push_one(const PushArgs& P, const Hist<FP>& H, uint32_t n, uint32_t w) {
    if (std::is_same<AT, float>::value && P.lut_meta) {
        uint32_t off, len, k;
        lut_row(P, n, w, off, len, k);
        if (len) {
            for (uint32_t e = 0; e < len; e++) {
                const uint2 ent = __ldg(P.lut + off + e);
                H.add_int(ent.x, k * ent.y);
            }
            return;
        }
    }
    if constexpr (FP) push_frac<AT>(P, H, n, (float)w);
    else push_int<FP>(P, H, n, w);
}

__device__ __forceinline__ uint32_t read_id(const Geom& G, const Ids& I, int l, int c, uint32_t idx) {
    if (l == 0)
        return G.id0_bytes == 2 ? (uint32_t)__ldg(static_cast<const uint16_t*>(I.l0[c]) + idx)
                                : __ldg(static_cast<const uint32_t*>(I.l0[c]) + idx);
    return __ldg(I.hi[c] + G.off[l][c] + idx);
}

// node ID of cube o of block B
__device__ __forceinline__ uint32_t cube_node(const Geom& G, const Ids& I, const Blk& B, uint32_t o, int& l) {
    l = B.meta & 31;
    const int c = (B.meta >> 5) & 3, e0 = (B.meta >> 7) & 31, e1 = (B.meta >> 12) & 31;
    const uint32_t f = o & ((1u << e0) - 1u);
    const uint32_t sc = (o >> e0) & ((1u << e1) - 1u);
    const uint32_t t = o >> (e0 + e1);
    return read_id(G, I, l, c, B.base + f + sc * G.st1[l][c] + t * G.st2[l][c]);
}

// one warp-aggregated contribution of cube node `id` at level l
template <bool FP, typename AT>
__device__ __forceinline__ void accumulate(const PushArgs& P, const Hist<FP>& H, bool valid, uint32_t id, int l) {
    const uint64_t key = valid ? ((uint64_t)l << 32 | id) : ~0ull;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (!valid || lane != __ffs(peers) - 1) return;
    const uint32_t W = (uint32_t)__popc(peers) << (3 * l);
    if (id < P.S) {
        H.add_int(id, W);
        return;
    }
    push_one<FP, AT>(P, H, id, W);
}

template <bool FP>
__device__ __forceinline__ Hist<FP> carve(uint8_t* smem, uint32_t S, uint32_t* ntouched) {
    Hist<FP> H;
    H.h = reinterpret_cast<uint32_t*>(smem);
    H.hf = FP ? reinterpret_cast<float*>(H.h + S) : nullptr;
    H.touched = reinterpret_cast<uint16_t*>(FP ? reinterpret_cast<uint8_t*>(H.hf + S)
                                               : reinterpret_cast<uint8_t*>(H.h + S));
    H.ntouched = ntouched;
    H.track = S > kScanFlushMax;
    return H;
}

template <bool FP>
__device__ __forceinline__ void flush(const Hist<FP>& H, uint32_t S, int64_t q, uint32_t* __restrict__ acc,
                                      float* __restrict__ accf) {
    // With the fp32 push a bin can be listed twice (once when its integer part
    // and once when its fractional part became non-zero), so bins are read and
    // cleared in one atomic step: the second reader sees zero.
    if (!H.track) {
        for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
            const uint32_t v = H.h[s];
            if (v) {
                H.h[s] = 0;
                atomicAdd(acc + q * S + s, v);
            }
            if constexpr (FP) {
                const float f = H.hf[s];
                if (f != 0.f) {
                    H.hf[s] = 0.f;
                    atomicAdd(accf + q * S + s, f);
                }
            }
        }
        return;
    }
    const uint32_t n = *H.ntouched;
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint32_t s = H.touched[t];
        const uint32_t v = FP ? atomicExch(H.h + s, 0u) : H.h[s];
        if (!FP) H.h[s] = 0;
        if (v) atomicAdd(acc + q * S + s, v);
        if constexpr (FP) {
            const float f = atomicExch(H.hf + s, 0.f);
            if (f != 0.f) atomicAdd(accf + q * S + s, f);
        }
    }
}

struct MainArgs {
    Geom G;
    Ids I;
    PushArgs P;
    const Blk* blk;
    const uint64_t* blk_off;
    const uint64_t* ncube;
    const uint64_t* chunk_off;
    const uint32_t* chunk_q;     // box of every chunk
    const uint32_t* chunk_b;     // block holding every chunk's first cube
    unsigned long long total_chunks;
    Lim lim;                     // device-side batch size (plans)
    int64_t Q;
    uint32_t chunk;
    unsigned long long* ticket;
    uint32_t* acc;
    float* accf;
    void* const* io;             // plans: io[1] is the output (acc for u32, accf for fp32)
    uint32_t qcap;               // entries of each warp's push queue (set by launch_main)
};

// the output a main kernel accumulates into: fixed, or (plans) the caller's
// buffer named in the plan's io slots
template <bool FP>
__device__ __forceinline__ void main_out(const MainArgs& A, uint32_t*& acc, float*& accf) {
    acc = A.acc;
    accf = A.accf;
    if (A.io) {
        if constexpr (FP) accf = static_cast<float*>(A.io[1]);
        else acc = static_cast<uint32_t*>(A.io[1]);
    }
}

// A warp's pending internal-node pushes: the unit loop appends (node, weight)
// to a queue in shared memory, and the queue is pushed 32 entries at a time
// (a measured alternative that summed the entries of one node in a hash
// table first was slower on every workload: its probes cost more than the
// expansions it saved).
// The queue is drained once it holds 32 entries; a step of the unit loop can
// add up to 8 per lane, and an entry that finds the queue full is pushed by
// its own lane at once (divergent, slower).  The launch takes the long queue
// unless a short one fits more CTAs on an SM: the loop is bound by load
// latency, so resident warps count for more where shared memory limits them.
constexpr uint32_t kQueueLong = 320, kQueueShort = 64;   // entries
constexpr size_t queue_bytes(uint32_t cap) { return (size_t)cap * 8 + 16; }   // nodes, weights, counter
constexpr size_t kMaxDynSmem = 227 * 1024;   // dynamic shared memory of one CTA at most

// chunks of the launch: known on the host, or (plans) read on the device,
// zero when the batch overflows the plan's buffers
__device__ __forceinline__ unsigned long long main_total(const MainArgs& A) {
    if (!A.lim.Qd) return A.total_chunks;
    const int64_t Qe = *A.lim.Qd;
    return over_cap(A.lim, A.blk_off, A.chunk_off, Qe) ? 0ull : A.chunk_off[Qe];
}

struct Queue {
    uint32_t* n;       // queued nodes
    uint32_t* w;       // queued weights
    uint32_t* count;   // queued entries
    uint32_t cap;      // room
};

__device__ __forceinline__ Queue carve_queue(uint8_t* p, uint32_t cap) {
    Queue Qu;
    Qu.n = reinterpret_cast<uint32_t*>(p);
    Qu.w = Qu.n + cap;
    Qu.count = Qu.w + cap;
    Qu.cap = cap;
    return Qu;
}

// empty queue (one warp)
__device__ __forceinline__ void clear_queue(const Queue& Qu) {
    if ((threadIdx.x & 31) == 0) *Qu.count = 0u;
    __syncwarp();
}

// push one (node, weight) per lane where `valid`.  With the mixture table each
// lane adds the first two entries of its node's row itself (rows average about
// two entries: two independent loads right after the row header); the rest of
// longer rows is flattened: entry e goes to lane e % 32, which finds its row by
// a binary search over the inclusive sums of the remaining lengths.  Nodes
// without a row (and 16-bit weights) walk their lerp trees.
template <bool FP, typename AT>
__device__ __forceinline__ void push_lanes(const PushArgs& P, const Hist<FP>& H, bool valid, uint32_t n,
                                           uint32_t w) {
    const int lane = threadIdx.x & 31;
    if (std::is_same<AT, float>::value && P.lut_meta) {
        uint32_t off = 0, len = 0, k = 0;
        if (valid) {
            lut_row(P, n, w, off, len, k);
            if (!len) {
                if constexpr (FP) push_frac<AT>(P, H, n, (float)w);
                else push_int<FP>(P, H, n, w);
            }
        }
        __syncwarp();
        if (len) {
            const uint2 e0 = __ldg(P.lut + off);
            const uint2 e1 = len > 1 ? __ldg(P.lut + off + 1) : make_uint2(0u, 0u);
            H.add_int(e0.x, k * e0.y);
            if (len > 1) H.add_int(e1.x, k * e1.y);
            const uint32_t h = len > 1 ? 2u : 1u;
            off += h;
            len -= h;
        }
        if (!__any_sync(0xffffffffu, len != 0u)) {
            __syncwarp();
            return;
        }
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - len;
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t e = base + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t v = __shfl_sync(0xffffffffu, incl, j + step - 1);
                if (v <= e) j += step;
            }
            const uint32_t oj = __shfl_sync(0xffffffffu, off, j);
            const uint32_t kj = __shfl_sync(0xffffffffu, k, j);
            const uint32_t ej = __shfl_sync(0xffffffffu, excl, j);
            if (e < total) {
                const uint2 ent = __ldg(P.lut + oj + (e - ej));
                H.add_int(ent.x, kj * ent.y);
            }
        }
    } else if (valid) {
        if constexpr (FP) push_frac<AT>(P, H, n, (float)w);
        else push_int<FP>(P, H, n, w);
    }
    __syncwarp();
}

// push queued entries 32 at a time until fewer than 32 (none if `all`)
// remain, then move the rest to the front.  Inlined: as a call it made the
// main loop save and restore its live registers around every drain (100,000-box
// batch 5.79 -> 5.48 ms)
template <bool FP, typename AT>
__device__ __forceinline__ void drain(const PushArgs& P, const Hist<FP>& H, const Queue& Qu, bool all) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t qc = min(*Qu.count, Qu.cap);   // entries past the end were pushed at once
    uint32_t done = 0;
    while (qc - done >= 32 || (all && qc > done)) {
        const uint32_t take = min(qc - done, 32u);
        const bool v = (uint32_t)lane < take;
        push_lanes<FP, AT>(P, H, v, v ? Qu.n[done + lane] : 0u, v ? Qu.w[done + lane] : 0u);
        done += take;
    }
    const uint32_t rest = qc - done;
    uint32_t tn = 0, tw = 0;
    if ((uint32_t)lane < rest) {
        tn = Qu.n[done + lane];
        tw = Qu.w[done + lane];
    }
    __syncwarp();
    if ((uint32_t)lane < rest) {
        Qu.n[lane] = tn;
        Qu.w[lane] = tw;
    }
    if (lane == 0) *Qu.count = rest;
    __syncwarp();
}

// Cubes [w0, w1) of one box by one warp, b the block holding cube w0.
//
// The span is a flat stream of units.  A window holds the records of 31
// consecutive blocks, one per lane; the part of each block inside the span is
// cut into units -- 32-byte vectors of IDs (16 uint16 or 8 uint32 of one row)
// where the block's rows are 32-byte aligned and at least that long, else
// 16-byte vectors where they are 16-byte aligned (Algorithm 1's runs start on
// multiples of their own length, so whole rows are), and single cubes for the
// unaligned head and tail and for every other block -- and a warp scan of
// the unit counts lets lane k find the block of unit u from a ballot of
// the block ends.
// Each lane takes units u, u + 32, ... (a 32-byte unit is two 16-byte loads),
// so no load waits on a block boundary.  Every lane keeps a run (level, node, count) of
// its own consecutive cubes; a finished run of a source is added to the
// shared histogram, one of an internal node (levels >= 1) is queued for the
// warp's pushes.
// RN: units per lane per step in windows without 32-byte units (2 in the
// per-warp kernel, whose registers are capped for occupancy; 4 in the CTA
// kernel, which has registers to spare: measured 4.67 -> 4.34 ms on the
// cylinder batch, while the per-warp kernel spills at 4)
template <bool FP, typename AT, int RN>
__device__ __forceinline__ void process_span(const MainArgs& A, const Hist<FP>& H, const Queue& Qu, uint32_t w0,
                                             uint32_t w1, uint64_t b, uint64_t b1, uint32_t ncube) {
    const int lane = threadIdx.x & 31;
    const uint32_t S = A.P.S;
    const int lg0 = A.G.id0_bytes == 2 ? 3 : 2;   // log2 level-0 IDs per 16 bytes
    uint32_t rid = kNone, rcnt = 0;
    int rl = 0;
    auto finish = [&]() {
        if (!rcnt) return;
        const uint32_t W = rcnt << (3 * rl);
        if (rl == 0 || rid < S) {
            H.add_int(rid, W);
        } else {
            const uint32_t pos = atomicAdd(Qu.count, 1u);
            if (pos < Qu.cap) {
                Qu.n[pos] = rid;
                Qu.w[pos] = W;
            } else {
                push_one<FP, AT>(A.P, H, rid, W);
            }
        }
    };
    auto feed = [&](uint32_t x, int l, uint32_t n = 1) {
        if (x == rid && l == rl) {
            rcnt += n;
        } else {
            finish();
            rid = x;
            rl = l;
            rcnt = n;
        }
    };
    for (uint64_t bb = b;; bb += 31) {
        const uint64_t i = bb + lane;
        uint32_t st = ncube, base = 0, meta = 0;
        if (i < b1) {
            const Blk t = A.blk[i];
            st = t.start;
            base = t.base;
            meta = t.meta;
        }
        const uint32_t nxt = __shfl_down_sync(0xffffffffu, st, 1);
        const uint32_t lo_a = max(st, w0), hi_a = min(nxt, w1);
        const bool use = lane < 31 && lo_a < hi_a;
        const int l = meta & 31, cp = (meta >> 5) & 3, e0 = (meta >> 7) & 31;
        // 32-byte units where the block's rows allow them, else 16-byte ones
        const int lg16 = l == 0 ? lg0 : 2;
        const uint32_t lo = use ? lo_a - st : 0u, hi = use ? hi_a - st : 0u;
        const bool wide = use && e0 > lg16 && ((A.G.vec32_ok[cp] >> l) & 1u) && hi - lo >= (4u << lg16);
        const int lg = lg16 + (wide ? 1 : 0);
        const bool vec = use && e0 >= lg && ((A.G.vec_ok[cp] >> l) & 1u) && hi - lo >= (2u << lg);
        const uint32_t vm = (1u << lg) - 1u;
        // scalar head [lo, ha), vectors [ha, hb), scalar tail [hb, hi)
        const uint32_t ha = vec ? (lo + vm) & ~vm : hi;
        const uint32_t hb = vec ? hi & ~vm : hi;
        const uint32_t nh = ha - lo, nv = (hb - ha) >> lg;
        const uint32_t units = use ? (hi - lo) - (hb - ha) + nv : 0u;
        const uint32_t wmeta = meta | (wide ? 1u << 22 : 0u);
        uint32_t incl = units;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - units;
        // R units per lane per step: one (16- or 32-byte) where the window
        // has 32-byte units, else RN, so scalar-heavy windows keep several
        // loads in flight per lane
        auto run_units = [&](auto rc) {
            constexpr int R = decltype(rc)::value;
            for (uint32_t u0 = 0; u0 < total; u0 += 32u * R) {
                uint4 va[R], vb[R];
                int kind[R], ul[R];   // kind: 0 scalar; 1 / 3: 4 / 8 uint32; 2 / 4: 8 / 16 uint16
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const uint32_t ub = u0 + 32u * r, u = ub + lane;
                    // block of unit u: blocks ending at or before ub, plus those
                    // ending inside this group at or before u (block ends are
                    // distinct below the total, so one bit each)
                    const unsigned below = __ballot_sync(0xffffffffu, incl <= ub);
                    const uint32_t te = incl - ub;
                    const unsigned ends = __reduce_or_sync(0xffffffffu, incl > ub && te < 32u ? 1u << te : 0u);
                    const int j = __popc(below) + __popc(ends & ((2u << lane) - 1u) & ~1u);
                    const uint32_t jbase = __shfl_sync(0xffffffffu, base, j & 31);
                    const uint32_t jmeta = __shfl_sync(0xffffffffu, wmeta, j & 31);
                    const uint32_t jlo = __shfl_sync(0xffffffffu, lo, j & 31);
                    const uint32_t jnh = __shfl_sync(0xffffffffu, nh, j & 31);
                    const uint32_t jnv = __shfl_sync(0xffffffffu, nv, j & 31);
                    const uint32_t jex = __shfl_sync(0xffffffffu, excl, j & 31);
                    kind[r] = -1;
                    ul[r] = 0;
                    va[r] = make_uint4(0u, 0u, 0u, 0u);
                    vb[r] = va[r];
                    if (u < total) {
                        const int jl = jmeta & 31, jc = (jmeta >> 5) & 3;
                        const int je0 = (jmeta >> 7) & 31, je1 = (jmeta >> 12) & 31;
                        const bool jw = R == 1 && ((jmeta >> 22) & 1u);
                        const int jlg = (jl == 0 ? lg0 : 2) + (jw ? 1 : 0);
                        const uint32_t t = u - jex;
                        uint32_t o;
                        bool vv = false;
                        if (t < jnh) {
                            o = jlo + t;
                        } else if (t < jnh + jnv) {
                            o = jlo + jnh + ((t - jnh) << jlg);
                            vv = true;
                        } else {
                            o = jlo + jnh + (jnv << jlg) + (t - jnh - jnv);
                        }
                        const uint32_t idx = jbase + (o & ((1u << je0) - 1u)) +
                                             ((o >> je0) & ((1u << je1) - 1u)) * A.G.st1[jl][jc] +
                                             (o >> (je0 + je1)) * A.G.st2[jl][jc];
                        ul[r] = jl;
                        const bool u16 = jl == 0 && lg0 == 3;
                        // IDs are read once: streaming loads (evict first) leave L2
                        // to the mixture table and node records the pushes gather
                        const void* row =
                            jl == 0 ? A.I.l0[jc] : static_cast<const void*>(A.I.hi[jc] + A.G.off[jl][jc]);
                        if (vv) {
                            const uint4* p = reinterpret_cast<const uint4*>(
                                u16 ? static_cast<const void*>(static_cast<const uint16_t*>(row) + idx)
                                    : static_cast<const void*>(static_cast<const uint32_t*>(row) + idx));
                            va[r] = __ldcs(p);
                            if (jw) vb[r] = __ldcs(p + 1);
                            kind[r] = (u16 ? 2 : 1) + (jw ? 2 : 0);
                        } else {
                            va[r].x = u16 ? (uint32_t)__ldcs(static_cast<const uint16_t*>(row) + idx)
                                          : __ldcs(static_cast<const uint32_t*>(row) + idx);
                            kind[r] = 0;
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int k = kind[r], l = ul[r];
                    const uint4 x = va[r], y = vb[r];
                    if (k == 0) {
                        feed(x.x, l);
                    } else if (k == 1 || k == 3) {
                        const bool same = rcnt && rl == l && x.x == rid && x.y == rid && x.z == rid && x.w == rid &&
                                          (k == 1 || (y.x == rid && y.y == rid && y.z == rid && y.w == rid));
                        if (same) {
                            rcnt += k == 1 ? 4 : 8;
                        } else {
                            feed(x.x, l);
                            feed(x.y, l);
                            feed(x.z, l);
                            feed(x.w, l);
                            if (k == 3) {
                                feed(y.x, l);
                                feed(y.y, l);
                                feed(y.z, l);
                                feed(y.w, l);
                            }
                        }
                    } else if (k == 2 || k == 4) {
                        // uniform vector (every ID equals the first): it extends
                        // the lane's run or starts a new one.  Mixed vector (a
                        // segment boundary inside): each ID is added to its bin
                        // at once -- level-0 IDs are bins, and the adds are
                        // independent where a run would chain them
                        const uint32_t a = x.x & 0xffffu, pa = a * 0x10001u;
                        uint32_t d = (x.x ^ pa) | (x.y ^ pa) | (x.z ^ pa) | (x.w ^ pa);
                        if (k == 4) d |= (y.x ^ pa) | (y.y ^ pa) | (y.z ^ pa) | (y.w ^ pa);
                        if (d == 0u) {
                            if (rcnt && rl == 0 && rid == a) {
                                rcnt += k == 2 ? 8 : 16;
                            } else {
                                finish();
                                rid = a;
                                rl = 0;
                                rcnt = k == 2 ? 8 : 16;
                            }
                        } else {
                            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                            for (int q = 0; q < 8; q++) H.add_int((w4[q >> 1] >> (16 * (q & 1))) & 0xffffu, 1u);
                            if (k == 4) {
                                const uint32_t x4[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                                for (int q = 0; q < 8; q++) H.add_int((x4[q >> 1] >> (16 * (q & 1))) & 0xffffu, 1u);
                            }
                        }
                    }
                }
                __syncwarp();
                if (*Qu.count >= 32) drain<FP, AT>(A.P, H, Qu, false);
            }
        };
        if (__any_sync(0xffffffffu, wide)) run_units(std::integral_constant<int, 1>{});
        else run_units(std::integral_constant<int, RN>{});
        const uint32_t st31 = __shfl_sync(0xffffffffu, st, 31);
        if (bb + 31 >= b1 || st31 >= w1) break;
    }
    finish();
    __syncwarp();
}

// Few segments: every warp owns a histogram in shared memory and takes whole
// chunks from the global ticket, so warps never wait for each other.
// Register budget by CTA size NT: 256 threads, at most 51 registers (5 CTAs
// per SM): the loop is bound by load latency, and 40 resident warps per SM
// beat 32 at 63 registers even with a few spilled values (0.40 vs 0.42 ms on
// the 10,000-box batch).  128 threads, at most 56 registers (9 CTAs): where
// shared memory holds 9-10 CTAs of 4 warps anyway (1,182 segments), fewer
// spills beat the tenth CTA (7.04 vs 7.25 ms on the 100,000-box batch; 64
// registers and 8 CTAs: 7.41 ms).
template <int NT> struct WarpKernelBounds;
template <> struct WarpKernelBounds<128> { static constexpr int min_ctas = 9; };
template <> struct WarpKernelBounds<256> { static constexpr int min_ctas = 5; };

template <bool FP, typename AT, int NT>
__global__ void __launch_bounds__(NT, WarpKernelBounds<NT>::min_ctas) query_warp_kernel(MainArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t S = A.P.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t hist_bytes = (size_t)S * 4 * (FP ? 2 : 1);
    uint8_t* mine = smem + warp * (hist_bytes + queue_bytes(A.qcap));
    Hist<FP> H;
    H.h = reinterpret_cast<uint32_t*>(mine);
    H.hf = FP ? reinterpret_cast<float*>(H.h + S) : nullptr;
    H.touched = nullptr;
    H.ntouched = nullptr;
    H.track = false;
    const Queue Qu = carve_queue(mine + hist_bytes, A.qcap);
    for (uint32_t i = lane; i < S; i += 32) {
        H.h[i] = 0;
        if constexpr (FP) H.hf[i] = 0.f;
    }
    clear_queue(Qu);
    grid_dependency_wait();
    uint32_t* acc;
    float* accf;
    main_out<FP>(A, acc, accf);
    const unsigned long long total = main_total(A);
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(A.ticket, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= total) break;
        const uint32_t q = __ldg(A.chunk_q + c);
        const uint32_t ncube = (uint32_t)A.ncube[q];
        const uint32_t c0 = (uint32_t)(c - A.chunk_off[q]) * A.chunk;
        const uint32_t c1 = min(c0 + A.chunk, ncube);
        process_span<FP, AT, 2>(A, H, Qu, c0, c1, __ldg(A.chunk_b + c), A.blk_off[q + 1], ncube);
        drain<FP, AT>(A.P, H, Qu, true);
        for (uint32_t s = lane; s < S; s += 32) {
            const uint32_t v = H.h[s];
            if (v) {
                H.h[s] = 0;
                atomicAdd(acc + (size_t)q * S + s, v);
            }
            if constexpr (FP) {
                const float f = H.hf[s];
                if (f != 0.f) {
                    H.hf[s] = 0.f;
                    atomicAdd(accf + (size_t)q * S + s, f);
                }
            }
        }
        __syncwarp();
    }
}

// Many segments: one histogram per CTA; the CTA takes a chunk and its warps
// take sub-spans of it (about two each) from a shared counter.
template <bool FP, typename AT>
__global__ void __launch_bounds__(512) query_batched_kernel(MainArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_ntouched;
    __shared__ unsigned long long s_chunk;
    __shared__ uint32_t s_q;
    __shared__ uint32_t s_next;
    const uint32_t S = A.P.S;
    const Hist<FP> H = carve<FP>(smem, S, &s_ntouched);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // per-warp queues follow the touched list
    const size_t touched_bytes = (size_t)S * 2 * (FP ? 2 : 1);
    uint8_t* qbase = reinterpret_cast<uint8_t*>(H.touched) + ((touched_bytes + 15) & ~(size_t)15);
    const Queue Qu = carve_queue(qbase + warp * queue_bytes(A.qcap), A.qcap);
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
        H.h[i] = 0;
        if constexpr (FP) H.hf[i] = 0.f;
    }
    if (threadIdx.x == 0) s_ntouched = 0;
    clear_queue(Qu);
    grid_dependency_wait();
    uint32_t* acc;
    float* accf;
    main_out<FP>(A, acc, accf);
    const unsigned long long total = main_total(A);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long c = atomicAdd(A.ticket, 1ull);
            s_chunk = c;
            s_next = 0;
            if (c < total) s_q = A.chunk_q[c];
        }
        __syncthreads();
        const unsigned long long c = s_chunk;
        if (c >= total) break;
        const uint32_t q = s_q;
        const uint32_t ncube = (uint32_t)A.ncube[q];
        const uint32_t c0 = (uint32_t)(c - A.chunk_off[q]) * A.chunk;
        const uint32_t c1 = min(c0 + A.chunk, ncube);
        const uint64_t b1 = A.blk_off[q + 1];
        const uint32_t sub = max(32u, (((c1 - c0) + 2 * nw - 1) / (2 * nw) + 31) & ~31u);
        uint64_t bhint = __ldg(A.chunk_b + c);   // a warp's sub-spans only move forward
        for (;;) {
            uint32_t k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
            if ((uint64_t)k * sub >= (uint64_t)(c1 - c0)) break;
            const uint32_t w0 = c0 + k * sub;
            const uint32_t w1 = min(w0 + sub, c1);
            uint64_t b = bhint;
            if (lane == 0) {   // block of the sub-span's first cube
                uint64_t lo = bhint, hi = b1;   // blk[lo].start <= w0 < blk[hi].start
                while (hi - lo > 1) {
                    const uint64_t mid = (lo + hi) >> 1;
                    if (__ldg(&A.blk[mid].start) <= w0) lo = mid;
                    else hi = mid;
                }
                b = lo;
            }
            b = __shfl_sync(0xffffffffu, b, 0);
            bhint = b;
            process_span<FP, AT, 4>(A, H, Qu, w0, w1, b, b1, ncube);
        }
        drain<FP, AT>(A.P, H, Qu, true);
        __syncthreads();
        flush<FP>(H, S, q, acc, accf);
        __syncthreads();
        if (threadIdx.x == 0) s_ntouched = 0;
    }
}

// Baseline (MG_SCHED_PLAIN): one launch per box, unbatched.  The launch has
// as many CTAs as the box's footprint needs (about 4,096 cubes each, at most
// a few per SM); CTA b walks the blocks in order and counts cubes
// [b * per_cta, (b + 1) * per_cta) of the box into its shared histogram, then
// adds it to the box's row.
template <bool FP, typename AT>
__global__ void __launch_bounds__(256) query_plain_kernel(MainArgs A, const int32_t* __restrict__ boxes, int64_t q,
                                                          uint32_t per_cta) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_ntouched;
    __shared__ Runs R;
    const uint32_t S = A.P.S;
    const Hist<FP> H = carve<FP>(smem, S, &s_ntouched);
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
        H.h[i] = 0;
        if constexpr (FP) H.hf[i] = 0.f;
    }
    int32_t b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
    if (!box_ok(b, A.G)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) set_status(A.P.status, kStatBadInput);
        return;
    }
    if (threadIdx.x == 0) {
        s_ntouched = 0;
        make_runs(b, A.G, R);
    }
    __syncthreads();
    const uint64_t c0 = (uint64_t)blockIdx.x * per_cta, c1 = c0 + per_cta;
    uint64_t start = 0;
    for (int k = 0; k < R.nz && start < c1; k++)
        for (int j = 0; j < R.ny && start < c1; j++)
            for (int i = 0; i < R.nx && start < c1; i++) {
                const uint32_t n = block_cubes(R.lx[i], R.ly[j], R.lz[k]);
                const uint64_t lo = max(start, c0), hi = min(start + n, c1);
                if (lo < hi) {
                    const Blk B = make_blk(A.G, 0, R.sx[i], R.sy[j], R.sz[k], R.lx[i], R.ly[j], R.lz[k]);
                    for (uint64_t base = lo - start; base < hi - start; base += blockDim.x) {
                        const uint32_t o = (uint32_t)base + threadIdx.x;
                        const bool valid = o < hi - start;
                        uint32_t id = 0;
                        int lv = 0;
                        if (valid) id = cube_node(A.G, A.I, B, o, lv);
                        accumulate<FP, AT>(A.P, H, valid, id, lv);
                    }
                }
                start += n;
            }
    __syncthreads();
    flush<FP>(H, S, q, A.acc, A.accf);
}

// Baseline (MG_SCHED_NAIVE): no footprint assembly, every level-0 voxel of
// the clipped box counted.  A box is read in the level-0 copy whose fastest
// axis is its longest side, so its rows are as long as its shape allows.  Its
// rows are cut into slabs of about kNaiveSlab voxels, taken from a global
// ticket by persistent CTAs; each CTA counts its slab into a shared histogram
// and adds it to the box's row.  A slab is one flat stream of (row, vector)
// slots, the 16-byte vectors (8 uint16 or 4 uint32 IDs) that its rows touch;
// each thread takes four consecutive slots per step (64 contiguous bytes) and
// keeps one run of equal IDs across them; a vector that is not uniform (or is
// cut by the row's ends) adds its in-row IDs one by one.  At most 51 registers
// (five CTAs of 256 threads per SM): the loop is bound by loads in flight
// (1,000 boxes of the 100,000-box recipe: 2.75 ms at 74 registers, 2.30 ms at
// 64, 2.13 ms at 51).
constexpr uint32_t kNaiveSlab = 1u << 16;

// the clipped box in the axis order of the copy it is read from: row length
// L along the copy's fastest axis, n1 rows along the second, n2 along the third
struct NaiveBox {
    int c;
    uint32_t L, n1, n2;
    uint32_t o0, o1, o2;   // origin in the copy's axis order
};
__device__ __forceinline__ NaiveBox naive_box(const int32_t* b, const Geom& G) {
    const uint32_t dx = (uint32_t)(min((int64_t)b[0] + b[3], (int64_t)G.dims[0][0]) - b[0]);
    const uint32_t dy = (uint32_t)(min((int64_t)b[1] + b[4], (int64_t)G.dims[0][1]) - b[1]);
    const uint32_t dz = (uint32_t)(min((int64_t)b[2] + b[5], (int64_t)G.dims[0][2]) - b[2]);
    NaiveBox B;
    if (dx >= dy && dx >= dz) {
        B = NaiveBox{0, dx, dy, dz, (uint32_t)b[0], (uint32_t)b[1], (uint32_t)b[2]};
    } else if (dy >= dz) {
        B = NaiveBox{1, dy, dz, dx, (uint32_t)b[1], (uint32_t)b[2], (uint32_t)b[0]};
    } else {
        B = NaiveBox{2, dz, dx, dy, (uint32_t)b[2], (uint32_t)b[0], (uint32_t)b[1]};
    }
    return B;
}
__device__ __forceinline__ uint32_t naive_rows_per(const NaiveBox& B) { return max(1u, kNaiveSlab / B.L); }

// slabs of every box (0 for a malformed box, whose row stays zero)
__global__ void naive_count_kernel(Geom G, const int32_t* __restrict__ boxes, int64_t Q, uint64_t* __restrict__ items,
                                   unsigned* __restrict__ status) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    int32_t b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
    if (!box_ok(b, G)) {
        set_status(status, kStatBadInput);
        items[q] = 0;
        return;
    }
    const NaiveBox B = naive_box(b, G);
    const uint64_t rows = (uint64_t)B.n1 * B.n2, per = naive_rows_per(B);
    items[q] = (rows + per - 1) / per;
}

template <bool FP, typename T>
__global__ void __launch_bounds__(256, 5) query_naive_kernel(Geom G, Ids I, const int32_t* __restrict__ boxes, int64_t Q,
                                                          const uint64_t* __restrict__ item_off,
                                                          unsigned long long* __restrict__ ticket,
                                                          uint32_t* __restrict__ acc, float* __restrict__ accf) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ unsigned long long s_item;
    uint32_t* h = reinterpret_cast<uint32_t*>(smem);
    const uint32_t S = G.S;
    constexpr int E = 16 / (int)sizeof(T);   // IDs per 16-byte vector
    const unsigned long long total = item_off[Q];
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) h[i] = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1ull);
        __syncthreads();
        const unsigned long long w = s_item;
        if (w >= total) break;
        int64_t lo = 0, hi = Q;   // item_off[lo] <= w < item_off[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= w) lo = mid;
            else hi = mid;
        }
        const int64_t q = lo;
        int32_t b[6];
#pragma unroll
        for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
        const NaiveBox B = naive_box(b, G);
        const int c = B.c;
        const T* ids = static_cast<const T*>(I.l0[c]);
        const uint64_t st1 = G.st1[0][c], st2 = G.st2[0][c];
        const int third = c == 0 ? 2 : c == 1 ? 0 : 1;   // the copy's third axis
        const uint64_t V0 = st2 * (uint64_t)G.dims[0][third];   // IDs in the copy's array
        const uint32_t per = naive_rows_per(B);
        const uint32_t r0 = (uint32_t)(w - item_off[q]) * per;
        const uint32_t r1 = (uint32_t)min((uint64_t)r0 + per, (uint64_t)B.n1 * B.n2);
        const uint32_t vpr = (B.L + E - 1) / E + 1;   // vectors a row of L IDs can touch
        const uint32_t nf = (r1 - r0) * vpr;          // <= 2^16 / E + 2^17, or one row of a longer box
        uint32_t rid = kNone, rcnt = 0;
        auto flush_run = [&]() {
            if (rcnt) atomicAdd(h + rid, rcnt);
        };
        for (uint32_t f0 = 4u * threadIdx.x; f0 < nf; f0 += 4u * blockDim.x) {
            // the first slot's row and vector; the others follow
            uint32_t row = f0 / vpr, vi = f0 - row * vpr;
            uint64_t e0 = 0;
            uint32_t rrow = kNone;
            uint4 u[4];
            uint64_t p0s[4], e0s[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                u[j] = make_uint4(0u, 0u, 0u, 0u);
                p0s[j] = ~0ull;
                e0s[j] = 0;
                if (f0 + j < nf) {
                    if (row != rrow) {
                        const uint32_t r = r0 + row, a2 = r / B.n1, a1 = r - a2 * B.n1;
                        e0 = (uint64_t)(B.o2 + a2) * st2 + (uint64_t)(B.o1 + a1) * st1 + B.o0;
                        rrow = row;
                    }
                    const uint64_t v = e0 / E + vi;
                    if (v * E < e0 + B.L) {
                        e0s[j] = e0;
                        p0s[j] = v * E;
                        if ((v + 1) * E <= V0) {
                            u[j] = __ldcs(reinterpret_cast<const uint4*>(ids) + v);
                        } else {   // the array's last vector, cut at its end
                            T* x = reinterpret_cast<T*>(&u[j]);
                            for (int k = 0; k < E && v * E + k < V0; k++) x[k] = __ldg(ids + v * E + k);
                        }
                    }
                }
                if (++vi == vpr) {
                    vi = 0;
                    row++;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint64_t p0 = p0s[j], e0j = e0s[j], e1 = e0j + B.L;
                if (p0 == ~0ull) continue;
                const uint4 x = u[j];
                uint32_t a, d;
                if (E == 8) {
                    a = x.x & 0xffffu;
                    const uint32_t pr = a * 0x10001u;
                    d = (x.x ^ pr) | (x.y ^ pr) | (x.z ^ pr) | (x.w ^ pr);
                } else {
                    a = x.x;
                    d = (x.y ^ a) | (x.z ^ a) | (x.w ^ a);
                }
                if (d == 0u && p0 >= e0j && p0 + E <= e1) {
                    if (rcnt && rid == a) {
                        rcnt += E;
                    } else {
                        flush_run();
                        rid = a;
                        rcnt = E;
                    }
                    continue;
                }
                // a mixed vector, or the cut end of a row: every in-row ID is
                // added to its bin at once (independent adds, no run chain)
                const int k0 = p0 < e0j ? (int)(e0j - p0) : 0;
                const int k1 = p0 + E > e1 ? (int)(e1 - p0) : E;
                const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int k = 0; k < E; k++)
                    if (k >= k0 && k < k1) atomicAdd(h + (uint32_t)xs[k], 1u);
            }
        }
        flush_run();
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
            const uint32_t cnt = h[i];
            if (cnt) {
                h[i] = 0;
                if (FP) atomicAdd(accf + q * S + i, (float)cnt);
                else atomicAdd(acc + q * S + i, cnt);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// finalisation
// ---------------------------------------------------------------------------
__global__ void dense_f32_rows_kernel(const uint32_t* __restrict__ acc, void* const* __restrict__ io,
                                      const int64_t* __restrict__ Qd, int64_t S) {
    float* out = static_cast<float*>(io[1]);
    const int64_t n = *Qd * S;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)acc[i] + out[i];
}

__global__ void dense_f32_kernel(const uint32_t* __restrict__ acc, float* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)acc[i] + out[i];
}

template <bool FP>
__global__ void csr_count_kernel(const uint32_t* __restrict__ acc, const float* __restrict__ accf, int64_t Q,
                                 uint32_t S, uint64_t* __restrict__ cnt) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= Q) return;
    uint64_t c = 0;
    for (uint32_t s = lane; s < S; s += 32) {
        bool nz = acc[q * S + s] != 0;
        if constexpr (FP) nz = nz || accf[q * S + s] != 0.f;
        c += nz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[q] = c;
}

template <bool FP>
__global__ void csr_write_kernel(const uint32_t* __restrict__ acc, const float* __restrict__ accf, int64_t Q,
                                 uint32_t S, const uint64_t* __restrict__ off, uint32_t* __restrict__ seg,
                                 void* __restrict__ out) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= Q) return;
    uint64_t pos = off[q];
    for (uint32_t sb = 0; sb < S; sb += 32) {
        const uint32_t s = sb + lane;
        uint32_t v = 0;
        float f = 0.f;
        bool nz = false;
        if (s < S) {
            v = acc[q * S + s];
            nz = v != 0;
            if constexpr (FP) {
                f = accf[q * S + s];
                nz = nz || f != 0.f;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) {
            const uint64_t o = pos + __popc(m & ((1u << lane) - 1u));
            seg[o] = s;
            if constexpr (FP) static_cast<float*>(out)[o] = (float)v + f;
            else static_cast<uint32_t*>(out)[o] = v;
        }
        pos += __popc(m);
    }
}

// box and first block of every chunk
// Exclusive scans of the per-box block and chunk counts for batches of up to
// kFusedScanMax boxes in one CTA: offsets[q] and the totals at [Q]; for plans
// the capacity check of the batch (entries past the live batch are zero).
constexpr int kScanThreads = 1024;
constexpr int64_t kFusedScanMax = 1 << 18;

__global__ void __launch_bounds__(kScanThreads) plan_scan_kernel(const uint32_t* __restrict__ nblk,
                                                                 const uint64_t* __restrict__ nchunk, int64_t Q,
                                                                 uint64_t* __restrict__ blk_off,
                                                                 uint64_t* __restrict__ chunk_off, Lim lim,
                                                                 unsigned* __restrict__ status) {
    __shared__ unsigned long long sb[32], sc[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned long long carry_b = 0, carry_c = 0;
    // tiles of kScanThreads consecutive boxes, one per thread (coalesced)
    for (int64_t t0 = 0; t0 < Q; t0 += kScanThreads) {
        const int64_t i = t0 + t;
        const unsigned long long xb = i < Q ? nblk[i] : 0ull, xc = i < Q ? nchunk[i] : 0ull;
        unsigned long long ib = xb, ic = xc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yb = __shfl_up_sync(0xffffffffu, ib, o);
            const unsigned long long yc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) {
                ib += yb;
                ic += yc;
            }
        }
        if (lane == 31) {
            sb[warp] = ib;
            sc[warp] = ic;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long wb = sb[lane], wc = sc[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long yb = __shfl_up_sync(0xffffffffu, wb, o);
                const unsigned long long yc = __shfl_up_sync(0xffffffffu, wc, o);
                if (lane >= o) {
                    wb += yb;
                    wc += yc;
                }
            }
            sb[lane] = wb;
            sc[lane] = wc;
        }
        __syncthreads();
        const unsigned long long pb = warp ? sb[warp - 1] : 0ull, pc = warp ? sc[warp - 1] : 0ull;
        if (i < Q) {
            blk_off[i] = carry_b + pb + ib - xb;
            chunk_off[i] = carry_c + pc + ic - xc;
        }
        carry_b += sb[31];
        carry_c += sc[31];
        __syncthreads();
    }
    if (t == 0) {
        blk_off[Q] = carry_b;
        chunk_off[Q] = carry_c;
        if (lim.Qd && (carry_b > lim.cap_blocks || carry_c > lim.cap_chunks)) set_status(status, kStatCapacity);
    }
}

// the live batch size of a plan run, passed by value (no host staging)
// and the caller's boxes and output named in the plan's io slots
__global__ void set_batch_kernel(int64_t* __restrict__ Qd, int64_t Q, void** __restrict__ io, const void* boxes,
                                 void* out) {
    *Qd = Q;
    io[0] = const_cast<void*>(boxes);
    io[1] = out;
}

// zero the first *Qd rows of S counters (plans); n = rows * S bound
template <typename T>
__global__ void zero_rows_kernel(T* __restrict__ a, const int64_t* __restrict__ Qd, int64_t S) {
    const int64_t n = *Qd * S;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = T(0);
}

__global__ void widen_kernel(const uint32_t* __restrict__ a, uint64_t* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

int sm_count(int dev) {
    static std::mutex mu;
    static std::vector<int> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev] ? cache[dev] : 1;
}

template <typename K>
mg_status prepare_kernel(K kernel, size_t smem) {
    MG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return MG_OK;
}

// pdl: launch the batched kernel with programmatic stream serialisation (its
// CTAs start while the plan kernel finishes and wait for it on the device)
template <bool FP, typename AT>
mg_status launch_main(const mg_graph* g, const MainArgs& A, const mg_query_opts& o, const int32_t* boxes,
                      size_t smem, int threads, cudaStream_t s, bool pdl = false, const Alloc* scratch = nullptr) {
    if (o.schedule == MG_SCHED_NAIVE) {
        // slabs per box, their offsets, then one persistent launch
        if (!scratch) return fail(MG_ERR_INVALID_ARG, "naive schedule without scratch");
        Buf items, off, ticket;
        MG_TRY(items.alloc(scratch, (size_t)A.Q * 8, s));
        MG_TRY(off.alloc(scratch, (size_t)(A.Q + 1) * 8, s));
        MG_TRY(ticket.alloc(scratch, 8, s));
        naive_count_kernel<<<grid_for(A.Q, 256), 256, 0, s>>>(A.G, boxes, A.Q, items.as<uint64_t>(), A.P.status);
        MG_CUDA(cudaGetLastError());
        MG_TRY(scan_exclusive_u64(items.as<uint64_t>(), off.as<uint64_t>(), A.Q, off.as<uint64_t>() + A.Q, *scratch,
                                  s));
        MG_CUDA(cudaMemsetAsync(ticket.p, 0, 8, s));
        const size_t sm = (size_t)g->S * 4;
        auto launch = [&](auto k) -> mg_status {
            MG_TRY(prepare_kernel(k, sm));
            int per_sm = 0;
            MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, sm));
            const int grid = std::max(per_sm, 1) * sm_count(g->device);
            k<<<grid, 256, sm, s>>>(A.G, A.I, boxes, A.Q, off.as<uint64_t>(), ticket.as<unsigned long long>(), A.acc,
                                    A.accf);
            MG_CUDA(cudaGetLastError());
            return MG_OK;
        };
        if (g->id0_bytes == 2) return launch(&query_naive_kernel<FP, uint16_t>);
        return launch(&query_naive_kernel<FP, uint32_t>);
    }
    if (o.schedule == MG_SCHED_PLAIN) {
        // footprint cubes of every box, read back to size each box's launch
        if (!scratch) return fail(MG_ERR_INVALID_ARG, "plain schedule without scratch");
        Buf cubes;
        MG_TRY(cubes.alloc(scratch, (size_t)A.Q * 8, s));
        plan_count_kernel<<<grid_for(A.Q * 32, kPlanThreads), kPlanThreads, 0, s>>>(
            A.G, boxes, A.Q, 1, nullptr, cubes.as<uint64_t>(), nullptr, A.P.status, Lim{nullptr, 0, 0});
        MG_CUDA(cudaGetLastError());
        std::vector<uint64_t> nc((size_t)A.Q);
        MG_CUDA(cudaMemcpyAsync(nc.data(), cubes.p, (size_t)A.Q * 8, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        auto k = query_plain_kernel<FP, AT>;
        MG_TRY(prepare_kernel(k, smem));
        const uint64_t max_ctas = 4ull * sm_count(g->device);
        for (int64_t q = 0; q < A.Q; q++) {
            const uint64_t n = std::max<uint64_t>(nc[q], 1);
            const uint64_t ctas = std::min<uint64_t>(max_ctas, (n + 4095) / 4096);
            const uint32_t per = (uint32_t)((n + ctas - 1) / ctas);
            k<<<(unsigned)ctas, 256, smem, s>>>(A, boxes, q, per);
        }
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    }
    // few segments: a private histogram per warp; else one per CTA (smem
    // is then the histogram's part, the warps' queues come on top)
    const int warps = threads / 32;
    const size_t hist_w = (size_t)g->S * 4 * (FP ? 2 : 1);
    const bool warp_mode =
        g->S <= kWarpHistMax && threads <= 256 && (hist_w + queue_bytes(kQueueShort)) * warps <= 96 * 1024;
    auto k = !warp_mode ? query_batched_kernel<FP, AT>
             : threads <= 128 ? query_warp_kernel<FP, AT, 128> : query_warp_kernel<FP, AT, 256>;
    auto smem_for = [&](uint32_t cap) {
        return warp_mode ? (hist_w + queue_bytes(cap)) * warps : smem + warps * queue_bytes(cap);
    };
    int per_sm = 0, per_long = 0;
    if (smem_for(kQueueShort) > kMaxDynSmem) return fail(MG_ERR_UNSUPPORTED, "query kernel does not fit on an SM");
    MG_TRY(prepare_kernel(k, smem_for(kQueueShort)));
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem_for(kQueueShort)));
    if (per_sm < 1) return fail(MG_ERR_UNSUPPORTED, "query kernel does not fit on an SM");
    if (smem_for(kQueueLong) <= kMaxDynSmem) {
        MG_TRY(prepare_kernel(k, smem_for(kQueueLong)));
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_long, k, threads, smem_for(kQueueLong)));
    }
    MainArgs A2 = A;
    A2.qcap = per_long >= per_sm ? kQueueLong : kQueueShort;
    const size_t sm = smem_for(A2.qcap);
    const int grid = per_sm * sm_count(g->device);
    if (!pdl) {
        k<<<grid, threads, sm, s>>>(A2);
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MG_CUDA(cudaLaunchKernelEx(&cfg, k, A2));
    return MG_OK;
}

// Box histograms summed from the mixture table (Sec. 3.6) with error bars
// (Sec. 3.5): one CTA per box walks its footprint blocks; every cube adds
// 8^l mu and (8^l dmu)^2 of each entry of its node's row into shared fp64
// accumulators; the row's error bars are the square roots.
__global__ void __launch_bounds__(256) query_lut_kernel(Geom G, Ids I, const int32_t* __restrict__ boxes,
                                                        const uint64_t* __restrict__ off,
                                                        const uint32_t* __restrict__ src, const double* __restrict__ mu,
                                                        const double* __restrict__ dmu, double* __restrict__ hist,
                                                        double* __restrict__ err, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ Runs R;
    const uint32_t S = G.S;
    double* h = reinterpret_cast<double*>(smem);
    double* e2 = h + S;
    const int64_t q = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < 2 * S; i += blockDim.x) h[i] = 0.0;
    int32_t b[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b[k] = boxes[q * 6 + k];
    const bool ok = box_ok(b, G);
    if (threadIdx.x == 0) {
        if (ok) make_runs(b, G, R);
        else set_status(status, kStatBadInput);
    }
    __syncthreads();
    if (ok) {
        // warps take the footprint's blocks in turn; a lane takes a contiguous
        // range of its block's cubes (consecutive cubes of a row) and keeps a
        // run of equal nodes, so a row of k cubes of node n at level l adds
        // k 8^l mu(n) and k (8^l dmu(n))^2 with one pass over n's row
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        const int nb = R.nx * R.ny * R.nz;
        uint32_t rn = 0xffffffffu, rc = 0;
        int rl = 0;
        auto flush_run = [&]() {
            if (!rc) return;
            const double W = ldexp((double)rc, 3 * rl), W2 = ldexp((double)rc, 6 * rl);
            for (uint64_t t = off[rn]; t < off[rn + 1]; t++) {
                const uint32_t s = src[t];
                if (s >= S) continue;
                atomicAdd(h + s, W * mu[t]);
                const double x = dmu[t];
                if (x != 0.0) atomicAdd(e2 + s, W2 * x * x);
            }
        };
        for (int bi = warp; bi < nb; bi += nwarps) {
            const int i = bi % R.nx, j = (bi / R.nx) % R.ny, k = bi / (R.nx * R.ny);
            const Blk B = make_blk(G, 0, R.sx[i], R.sy[j], R.sz[k], R.lx[i], R.ly[j], R.lz[k]);
            const uint32_t n = block_cubes(R.lx[i], R.ly[j], R.lz[k]);
            const uint32_t per = (n + 31) / 32, o0 = min(n, lane * per), o1 = min(n, o0 + per);
            for (uint32_t o = o0; o < o1; o++) {
                int lv = 0;
                const uint32_t node = cube_node(G, I, B, o, lv);
                if (node == rn && lv == rl) {
                    rc++;
                } else {
                    flush_run();
                    rn = node;
                    rl = lv;
                    rc = 1;
                }
            }
        }
        flush_run();
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        hist[q * S + s] = h[s];
        if (err) err[q * S + s] = sqrt(e2[s]);
    }
}

}  // namespace

mg_status query_lut(const mg_graph* g, const int32_t* boxes, int64_t Q, double* hist, double* err, cudaStream_t s) {
    if (!g->err_off.p) return fail(MG_ERR_INVALID_ARG, "build the mixture table first (mg_error_table_build)");
    const size_t sm = (size_t)g->S * 16;
    if (sm > 200 * 1024) return fail(MG_ERR_UNSUPPORTED, "too many segments for the shared fp64 accumulators");
    if (Q == 0) return MG_OK;
    MG_CUDA(cudaFuncSetAttribute(query_lut_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    query_lut_kernel<<<(unsigned)Q, 256, sm, s>>>(make_geom(g), make_ids(g), boxes, g->err_off.as<uint64_t>(),
                                                   g->err_src.as<uint32_t>(), g->err_mu.as<double>(),
                                                   g->err_dmu.as<double>(), hist, err, g->status.as<unsigned>());
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status count_cubes(const mg_graph* g, const int32_t* boxes, int64_t Q, uint64_t* cubes, cudaStream_t s) {
    const Geom G = make_geom(g);
    plan_count_kernel<<<grid_for(Q * 32, kPlanThreads), kPlanThreads, 0, s>>>(G, boxes, Q, 1, nullptr, cubes, nullptr,
                                                            g->status.as<unsigned>(), Lim{nullptr, 0, 0});
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

namespace {

// Scratch comes from `al`; `words` are two host words for readbacks; `room`,
// when not null, returns the bytes `al` can still hand out (fixed pools).
mg_status query_boxes_impl(const mg_graph* g, const int32_t* boxes, int64_t Q, const mg_query_opts& o, void* out,
                           size_t cap, uint32_t* seg, uint64_t* offsets, size_t* required, cudaStream_t s,
                           const Alloc& al, uint64_t* words, size_t (*room)(const Alloc&)) {
    const uint32_t S = g->S;
    const bool FP = o.hist_type == MG_HIST_F32;
    const bool csr = o.layout == MG_LAYOUT_CSR;
    if (S > kMaxSharedSegments) return fail(MG_ERR_UNSUPPORTED, "more than 32768 segments");
    if (required) *required = 0;
    if (Q == 0) {
        if (csr) MG_CUDA(cudaMemsetAsync(offsets, 0, sizeof(uint64_t), s));
        return MG_OK;
    }
    if (FP && o.alpha_dtype != MG_F32) MG_TRY(ensure_alpha16(const_cast<mg_graph*>(g), (mg_dtype)o.alpha_dtype, s));
    const int tuned_c = g->tuned_chunk[FP ? 1 : 0], tuned_t = g->tuned_threads[FP ? 1 : 0];
    const uint32_t chunk = o.chunk_cubes > 0 ? (uint32_t)o.chunk_cubes : tuned_c > 0 ? (uint32_t)tuned_c : 2048u;
    const int threads = o.block_threads > 0 ? o.block_threads : tuned_t > 0 ? tuned_t : 256;
    const Geom G = make_geom(g);
    unsigned* status = g->status.as<unsigned>();
    mg_graph* gm = const_cast<mg_graph*>(g);
    const bool timed = o.timing != 0;
    if (timed) {
        for (auto& e : gm->qev)
            if (!e) MG_CUDA(cudaEventCreate(&e));
        gm->qev_valid = false;
        MG_CUDA(cudaEventRecord(gm->qev[0], s));
    }

    // accumulators: the dense u32 output itself, else scratch
    Buf acc_b, accf_b;
    uint32_t* acc = nullptr;
    float* accf = nullptr;
    const size_t cells = (size_t)Q * S;
    if (!csr && !FP) {
        acc = static_cast<uint32_t*>(out);
    } else {
        MG_TRY(acc_b.alloc(&al, cells * 4, s));
        acc = acc_b.as<uint32_t>();
    }
    if (FP) {
        if (!csr) {
            accf = static_cast<float*>(out);
        } else {
            MG_TRY(accf_b.alloc(&al, cells * 4, s));
            accf = accf_b.as<float>();
        }
    }

    MainArgs A;
    A.G = G;
    A.I = make_ids(g);
    A.P.pq = g->pq.as<uint2>();
    A.P.ab32 = g->ab32.as<uint2>();
    A.P.lut_meta = g->lut_meta.as<uint2>();
    A.P.lut = g->lut.as<uint2>();
    A.P.alpha = o.alpha_dtype == MG_F16 ? g->alpha16.p : o.alpha_dtype == MG_BF16 ? g->alphab16.p : g->alpha.p;
    A.P.S = S;
    A.P.status = status;
    A.Q = Q;
    A.chunk = chunk;
    A.acc = acc;
    A.accf = accf;
    A.blk = nullptr;
    A.blk_off = nullptr;
    A.ncube = nullptr;
    A.chunk_off = nullptr;
    A.chunk_q = nullptr;
    A.chunk_b = nullptr;
    A.total_chunks = 0;
    A.lim = Lim{nullptr, 0, 0};
    A.ticket = nullptr;
    A.io = nullptr;
    A.qcap = kQueueShort;

    const size_t touched_bytes = (size_t)S * 2 * (FP ? 2 : 1);
    const size_t smem = (size_t)S * 4 * (FP ? 2 : 1) + ((touched_bytes + 15) & ~(size_t)15) + 16;
    if (smem > 220 * 1024) return fail(MG_ERR_UNSUPPORTED, "too many segments for the shared-memory histogram");
    Buf nblk, ncube, nchunk, blk_off, chunk_off, blk, ticket, chunk_q, chunk_b;
    if (o.schedule == MG_SCHED_BATCHED) {
        MG_TRY(nblk.alloc(&al, (size_t)Q * 4, s));
        MG_TRY(ncube.alloc(&al, (size_t)Q * 8, s));
        MG_TRY(nchunk.alloc(&al, (size_t)Q * 8, s));
        MG_TRY(blk_off.alloc(&al, (size_t)(Q + 1) * 8, s));
        MG_TRY(chunk_off.alloc(&al, (size_t)(Q + 1) * 8, s));
        MG_TRY(ticket.alloc(&al, 8, s));
        plan_count_kernel<<<grid_for(Q * 32, kPlanThreads), kPlanThreads, 0, s>>>(G, boxes, Q, chunk, nblk.as<uint32_t>(),
                                                                ncube.as<uint64_t>(), nchunk.as<uint64_t>(),
                                                                status, Lim{nullptr, 0, 0});
        MG_CUDA(cudaGetLastError());
        if (Q <= kFusedScanMax) {
            plan_scan_kernel<<<1, kScanThreads, 0, s>>>(nblk.as<uint32_t>(), nchunk.as<uint64_t>(), Q,
                                                        blk_off.as<uint64_t>(), chunk_off.as<uint64_t>(),
                                                        Lim{nullptr, 0, 0}, status);
            MG_CUDA(cudaGetLastError());
        } else {
            // block offsets are 64-bit sums of the 32-bit per-box counts
            MG_TRY(scan_exclusive_u64(nchunk.as<uint64_t>(), chunk_off.as<uint64_t>(), Q,
                                      chunk_off.as<uint64_t>() + Q, al, s));
            Buf nb64;
            MG_TRY(nb64.alloc(&al, (size_t)Q * 8, s));
            widen_kernel<<<grid_for(Q, 256, 152 * 64), 256, 0, s>>>(nblk.as<uint32_t>(), nb64.as<uint64_t>(), Q);
            MG_CUDA(cudaGetLastError());
            MG_TRY(scan_exclusive_u64(nb64.as<uint64_t>(), blk_off.as<uint64_t>(), Q, blk_off.as<uint64_t>() + Q, al,
                                      s));
        }
        uint64_t* totals = words;   // blocks, chunks
        MG_CUDA(cudaMemcpyAsync(&totals[0], blk_off.as<uint64_t>() + Q, 8, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaMemcpyAsync(&totals[1], chunk_off.as<uint64_t>() + Q, 8, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        if (totals[0] >= (1ull << 32) || totals[1] >= (1ull << 32))
            return fail(MG_ERR_UNSUPPORTED, "more than 2^32 footprint blocks or work chunks in one call");
        if (room) {
            const size_t need = (((size_t)std::max<uint64_t>(totals[0], 1) * sizeof(Blk) + 255) & ~(size_t)255) +
                                2 * (((size_t)std::max<uint64_t>(totals[1], 1) * 4 + 255) & ~(size_t)255);
            if (need > room(al))
                return fail(MG_ERR_CAPACITY, "these boxes need " + std::to_string(need >> 10) +
                                                 " KiB of footprint scratch; " + std::to_string(room(al) >> 10) +
                                                 " KiB of the fixed scratch remain: split the batch");
        }
        MG_TRY(blk.alloc(&al, (size_t)std::max<uint64_t>(totals[0], 1) * sizeof(Blk), s));
        MG_TRY(chunk_q.alloc(&al, (size_t)std::max<uint64_t>(totals[1], 1) * 4, s));
        MG_TRY(chunk_b.alloc(&al, (size_t)std::max<uint64_t>(totals[1], 1) * 4, s));
        plan_write_kernel<<<grid_for(Q * 32, kPlanThreads), kPlanThreads, 0, s>>>(
            G, boxes, Q, blk_off.as<uint64_t>(), blk.as<Blk>(), Lim{nullptr, 0, 0}, chunk_off.as<uint64_t>(), chunk,
            chunk_q.as<uint32_t>(), chunk_b.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
        A.chunk_q = chunk_q.as<uint32_t>();
        A.chunk_b = chunk_b.as<uint32_t>();
        A.total_chunks = totals[1];
        MG_CUDA(cudaMemsetAsync(ticket.p, 0, 8, s));
        A.blk = blk.as<Blk>();
        A.blk_off = blk_off.as<uint64_t>();
        A.ncube = ncube.as<uint64_t>();
        A.chunk_off = chunk_off.as<uint64_t>();
        A.ticket = ticket.as<unsigned long long>();
    }
    // the accumulators are cleared only once the footprint is known to fit, so
    // a refused call leaves the caller's output as it was
    if (FP) MG_CUDA(cudaMemsetAsync(accf, 0, cells * 4, s));
    MG_CUDA(cudaMemsetAsync(acc, 0, cells * 4, s));
    if (timed) MG_CUDA(cudaEventRecord(gm->qev[1], s));
    if (FP) {
        if (o.alpha_dtype == MG_F16)
            MG_TRY((launch_main<true, __half>(g, A, o, boxes, smem, threads, s, false, &al)));
        else if (o.alpha_dtype == MG_BF16)
            MG_TRY((launch_main<true, __nv_bfloat16>(g, A, o, boxes, smem, threads, s, false, &al)));
        else
            MG_TRY((launch_main<true, float>(g, A, o, boxes, smem, threads, s, false, &al)));
    } else {
        MG_TRY((launch_main<false, float>(g, A, o, boxes, smem, threads, s, false, &al)));
    }

    if (timed) MG_CUDA(cudaEventRecord(gm->qev[2], s));
    if (!csr) {
        if (FP) {
            dense_f32_kernel<<<grid_for((int64_t)cells, 256, 152 * 64), 256, 0, s>>>(acc, accf, (int64_t)cells);
            MG_CUDA(cudaGetLastError());
        }
        if (timed) {
            MG_CUDA(cudaEventRecord(gm->qev[3], s));
            gm->qev_valid = true;
        }
        return MG_OK;
    }
    // CSR: count, scan, capacity check, write
    Buf cnt;
    MG_TRY(cnt.alloc(&al, (size_t)Q * 8, s));
    if (FP)
        csr_count_kernel<true><<<grid_for(Q * 32, 256), 256, 0, s>>>(acc, accf, Q, S, cnt.as<uint64_t>());
    else
        csr_count_kernel<false><<<grid_for(Q * 32, 256), 256, 0, s>>>(acc, accf, Q, S, cnt.as<uint64_t>());
    MG_CUDA(cudaGetLastError());
    MG_TRY(scan_exclusive_u64(cnt.as<uint64_t>(), offsets, Q, offsets + Q, al, s));
    uint64_t* nnz_p = words;
    MG_CUDA(cudaMemcpyAsync(nnz_p, offsets + Q, 8, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    const uint64_t nnz = *nnz_p;
    if (required) *required = (size_t)nnz;
    if (nnz > cap) return fail(MG_ERR_CAPACITY, "CSR output needs " + std::to_string(nnz) + " entries");
    if (FP)
        csr_write_kernel<true><<<grid_for(Q * 32, 256), 256, 0, s>>>(acc, accf, Q, S, offsets, seg, out);
    else
        csr_write_kernel<false><<<grid_for(Q * 32, 256), 256, 0, s>>>(acc, accf, Q, S, offsets, seg, out);
    MG_CUDA(cudaGetLastError());
    if (timed) {
        MG_CUDA(cudaEventRecord(gm->qev[3], s));
        gm->qev_valid = true;
    }
    return MG_OK;
}

}  // namespace

mg_status query_boxes(const mg_graph* g, const int32_t* boxes, int64_t Q, const mg_query_opts& o, void* out,
                      size_t cap, uint32_t* seg, uint64_t* offsets, size_t* required, cudaStream_t s) {
    Arena* arena = nullptr;
    MG_TRY(arena_begin(const_cast<mg_graph*>(g), s, &arena));
    uint64_t local[2] = {0, 0};
    return query_boxes_impl(g, boxes, Q, o, out, cap, seg, offsets, required, s, arena->view,
                            arena->pinned ? arena->pinned : local, nullptr);
}

mg_status query_timing(const mg_graph* g, float* plan_ms, float* main_ms, float* out_ms) {
    if (!g->qev_valid) return fail(MG_ERR_INVALID_ARG, "no timed query call on this graph");
    MG_CUDA(cudaEventSynchronize(g->qev[3]));
    float t[3];
    for (int i = 0; i < 3; i++) MG_CUDA(cudaEventElapsedTime(&t[i], g->qev[i], g->qev[i + 1]));
    if (plan_ms) *plan_ms = t[0];
    if (main_ms) *main_ms = t[1];
    if (out_ms) *out_ms = t[2];
    return MG_OK;
}

}  // namespace mg

// ---------------------------------------------------------------------------
// Box histograms for callers that cannot allocate device memory: the same
// exact dense query with its scratch in a fixed array compiled into the
// library instead of memory from the allocator.
// ---------------------------------------------------------------------------
namespace mg {
namespace {

// Fixed scratch of mg_query_boxes_noalloc.  Every GPU that loads the library
// holds these 64 MiB until the process exits.
constexpr size_t kNoAllocBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};   // device address of the array, per device

// Host code only knows a stand-in for the array's name; the device address is
// looked up once per device, with that device current.
mg_status noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 256) return fail(MG_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fixed query scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return MG_OK;
}

// bump allocation from the fixed array for one call
struct Pool {
    unsigned char* base;
    size_t cap, used;
};

void* pool_alloc(void* ctx, size_t bytes, mg_stream) {
    Pool* pl = static_cast<Pool*>(ctx);
    const size_t n = (bytes + 255) & ~(size_t)255;
    if (pl->used + n > pl->cap) return nullptr;
    void* p = pl->base + pl->used;
    pl->used += n;
    return p;
}

void pool_free(void*, void*, size_t, mg_stream) {}

size_t pool_room(const Alloc& al) {
    const Pool* pl = static_cast<const Pool*>(al.a.ctx);
    return pl->cap - pl->used;
}

size_t rounded(size_t n) { return (n + 255) & ~(size_t)255; }

// scratch of the per-box plan arrays and their scans, before the footprint blocks
size_t per_box_scratch(int64_t Q) {
    const size_t q = (size_t)Q;
    const size_t parts = rounded(8 * ((q + 2047) / 2048)) * 2;   // one scan level's partial sums
    return rounded(4 * q) + 5 * rounded(8 * (q + 1)) + rounded(8) + 2 * (parts + 2 * rounded(8)) + 4096;
}

}  // namespace
}  // namespace mg

extern "C" MG_API mg_status mg_query_boxes_noalloc(const mg_graph* g, const int32_t* boxes, int64_t Q, uint32_t* out,
                                                   size_t out_capacity, mg_stream stream) {
    MG_RANGE("mg_query_boxes_noalloc");
    using namespace mg;
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (Q < 0) return fail(MG_ERR_INVALID_ARG, "Q must be >= 0");
    if (Q == 0) return MG_OK;
    if (!boxes || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if ((uint64_t)out_capacity < (uint64_t)Q * g->S) return fail(MG_ERR_INVALID_ARG, "out_capacity must be >= Q*S");
    if (g->S > kMaxSharedSegments) return fail(MG_ERR_UNSUPPORTED, "more than 32768 segments");
    if (g->quantised) return fail(MG_ERR_UNSUPPORTED, "a quantised graph has no exact weights");
    if (per_box_scratch(Q) > kNoAllocBytes / 2) {
        int64_t qmax = 1;
        while (per_box_scratch(qmax * 2) <= kNoAllocBytes / 2) qmax *= 2;
        return fail(MG_ERR_CAPACITY, "at most about " + std::to_string(qmax) +
                                         " boxes fit the fixed query scratch in one call: split the batch");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) MG_CUDA(cudaSetDevice(g->device));
    unsigned char* base = nullptr;
    mg_status st = noalloc_scratch(g->device, &base);
    if (st == MG_OK) {
        Pool pool{base, kNoAllocBytes, 0};
        Alloc al;
        al.a.ctx = &pool;
        al.a.alloc = pool_alloc;
        al.a.free = pool_free;
        al.custom = true;
        mg_query_opts o{};   // exact uint32 counts, dense, batched, default tuning
        uint64_t words[2] = {0, 0};
        st = query_boxes_impl(g, boxes, Q, o, out, out_capacity, nullptr, nullptr, nullptr,
                              reinterpret_cast<cudaStream_t>(stream), al, words, pool_room);
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return st;
}

// ---------------------------------------------------------------------------
// Query plans: the whole batched pipeline for up to max_Q boxes captured once
// as a CUDA graph, with every buffer preallocated; a run copies the boxes in,
// replays the graph and copies the histograms out, with no host sync.
// ---------------------------------------------------------------------------
struct mg_query_plan {
    mg_graph* g = nullptr;
    int64_t max_Q = 0;
    bool fp = false;
    uint32_t chunk = 0;
    int threads = 0;
    uint64_t cap_blocks = 0, cap_chunks = 0;
    mg::Buf pool;
    mg::Pool bump{nullptr, 0, 0};
    int32_t* boxes = nullptr;
    int64_t* Qd = nullptr;
    void* result = nullptr;   // max_Q x S, uint32 or fp32
    void** io = nullptr;      // device slots: the run's boxes and output (default: boxes, result)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool timed = false, ran = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // graph start, plan done, main done
    ~mg_query_plan() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace mg {
namespace {

template <bool FP, typename AT>
mg_status plan_enqueue(mg_query_plan* p, const Alloc& al, cudaStream_t s) {
    const mg_graph* g = p->g;
    const int64_t Q = p->max_Q;
    const uint32_t S = g->S;
    const Geom G = make_geom(g);
    unsigned* status = g->status.as<unsigned>();
    const Lim lim{p->Qd, p->cap_blocks, p->cap_chunks};
    Buf acc_b, ncube, blk_off, chunk_off, blk, chunk_q, chunk_b, tiles, ticket;
    uint32_t* acc = nullptr;
    float* accf = nullptr;
    if (FP) {
        MG_TRY(acc_b.alloc(&al, (size_t)Q * S * 4, s));
        acc = acc_b.as<uint32_t>();
        accf = static_cast<float*>(p->result);
    } else {
        acc = static_cast<uint32_t*>(p->result);
    }
    const int tb = tile_boxes(Q, sm_count(g->device));
    const int64_t ntiles = (Q + tb - 1) / tb;
    const int chunk_shift = (p->chunk & (p->chunk - 1)) == 0 ? __builtin_ctz(p->chunk) : -1;
    MG_TRY(ncube.alloc(&al, (size_t)Q * 8, s));
    MG_TRY(blk_off.alloc(&al, (size_t)(Q + 1) * 8, s));
    MG_TRY(chunk_off.alloc(&al, (size_t)(Q + 1) * 8, s));
    MG_TRY(blk.alloc(&al, (size_t)p->cap_blocks * sizeof(Blk), s));
    MG_TRY(chunk_q.alloc(&al, (size_t)p->cap_chunks * 4, s));
    MG_TRY(chunk_b.alloc(&al, (size_t)p->cap_chunks * 4, s));
    MG_TRY(tiles.alloc(&al, (size_t)ntiles * 16, s));
    MG_TRY(ticket.alloc(&al, 16, s));   // tile order, main-kernel chunks

    if (p->timed) MG_CUDA(cudaEventRecordWithFlags(p->ev[0], s, cudaEventRecordExternal));
    plan_reset_kernel<<<grid_for(2 * ntiles, 256, 152 * 4), 256, 0, s>>>(p->Qd, tb, tiles.as<uint64_t>(),
                                                                         ticket.as<unsigned long long>());
    MG_CUDA(cudaGetLastError());
    FusedOut F;
    F.ncube = ncube.as<uint64_t>();
    F.blk_off = blk_off.as<uint64_t>();
    F.chunk_off = chunk_off.as<uint64_t>();
    F.blk = blk.as<Blk>();
    F.chunk_q = chunk_q.as<uint32_t>();
    F.chunk_b = chunk_b.as<uint32_t>();
    F.tiles = tiles.as<uint64_t>();
    F.ticket = ticket.as<unsigned long long>();
    F.acc = acc;
    F.accf = accf;
    F.io = p->io;
    plan_fused_kernel<<<(unsigned)ntiles, kFusedThreads, 0, s>>>(G, p->boxes, Q, tb, p->chunk, chunk_shift, lim, F,
                                                                 status);
    MG_CUDA(cudaGetLastError());
    if (p->timed) MG_CUDA(cudaEventRecordWithFlags(p->ev[1], s, cudaEventRecordExternal));

    MainArgs A;
    A.G = G;
    A.I = make_ids(g);
    A.P.pq = g->pq.as<uint2>();
    A.P.ab32 = g->ab32.as<uint2>();
    A.P.lut_meta = g->lut_meta.as<uint2>();
    A.P.lut = g->lut.as<uint2>();
    A.P.alpha = std::is_same<AT, __half>::value ? g->alpha16.p : std::is_same<AT, __nv_bfloat16>::value ? g->alphab16.p
                                                                                                          : g->alpha.p;
    A.P.S = S;
    A.P.status = status;
    A.blk = blk.as<Blk>();
    A.blk_off = blk_off.as<uint64_t>();
    A.ncube = ncube.as<uint64_t>();
    A.chunk_off = chunk_off.as<uint64_t>();
    A.chunk_q = chunk_q.as<uint32_t>();
    A.chunk_b = chunk_b.as<uint32_t>();
    A.total_chunks = 0;
    A.lim = lim;
    A.Q = Q;
    A.chunk = p->chunk;
    A.ticket = ticket.as<unsigned long long>() + 1;
    A.acc = acc;
    A.accf = accf;
    A.io = p->io;
    A.qcap = kQueueShort;
    mg_query_opts o{};
    o.hist_type = FP ? MG_HIST_F32 : MG_HIST_U32;
    const size_t touched_bytes = (size_t)S * 2 * (FP ? 2 : 1);
    const size_t smem = (size_t)S * 4 * (FP ? 2 : 1) + ((touched_bytes + 15) & ~(size_t)15) + 16;
    MG_TRY((launch_main<FP, AT>(g, A, o, nullptr, smem, p->threads, s, !p->timed)));
    if (p->timed) MG_CUDA(cudaEventRecordWithFlags(p->ev[2], s, cudaEventRecordExternal));
    if (FP) {
        dense_f32_rows_kernel<<<grid_for(Q * S, 256, 152 * 64), 256, 0, s>>>(acc, p->io, p->Qd, S);
        MG_CUDA(cudaGetLastError());
    }
    return MG_OK;
}

}  // namespace
}  // namespace mg

namespace mg {
PlanParts plan_parts(const mg_query_plan* p) {
    return PlanParts{p->boxes, p->Qd, p->result, p->exec, p->chunk, p->cap_blocks, p->cap_chunks};
}
}  // namespace mg

using mg::fail;

extern "C" {

MG_API mg_status mg_query_plan_create(mg_graph* g, int64_t max_Q, const mg_query_opts* opts, int64_t max_blocks,
                                      int64_t max_chunks, mg_query_plan** out) {
    MG_RANGE("mg_query_plan_create");
    using namespace mg;
    if (!g || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (max_Q < 1 || max_Q >= (1ll << 31)) return fail(MG_ERR_INVALID_ARG, "max_Q must be in 1..2^31-1");
    if (max_blocks < 0 || max_chunks < 0) return fail(MG_ERR_INVALID_ARG, "negative capacity");
    mg_query_opts o{};
    if (opts) o = *opts;
    if (o.layout != MG_LAYOUT_DENSE || o.schedule != MG_SCHED_BATCHED)
        return fail(MG_ERR_UNSUPPORTED, "plans hold the dense layout and the batched schedule");
    if (o.hist_type != MG_HIST_U32 && o.hist_type != MG_HIST_F32) return fail(MG_ERR_INVALID_ARG, "bad hist_type");
    if (g->quantised && o.hist_type == MG_HIST_U32)
        return fail(MG_ERR_UNSUPPORTED, "a quantised graph has no exact weights: use MG_HIST_F32");
    if (o.alpha_dtype != MG_F32 && (o.hist_type == MG_HIST_U32 || (o.alpha_dtype != MG_F16 && o.alpha_dtype != MG_BF16)))
        return fail(MG_ERR_INVALID_ARG, "bad alpha_dtype");
    if (o.block_threads && o.block_threads != 128 && o.block_threads != 256 && o.block_threads != 512)
        return fail(MG_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
    if (o.chunk_cubes < 0) return fail(MG_ERR_INVALID_ARG, "negative chunk_cubes");
    if (g->S > kMaxSharedSegments) return fail(MG_ERR_UNSUPPORTED, "more than 32768 segments");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) MG_CUDA(cudaSetDevice(g->device));
    std::unique_ptr<mg_query_plan> p(new (std::nothrow) mg_query_plan());
    mg_status st = p ? MG_OK : fail(MG_ERR_OOM, "host allocation failed");
    if (st == MG_OK) {
        const bool FP = o.hist_type == MG_HIST_F32;
        p->g = g;
        p->max_Q = max_Q;
        p->fp = FP;
        const int tc = g->tuned_chunk[FP], tt = g->tuned_threads[FP];
        p->chunk = o.chunk_cubes > 0 ? (uint32_t)o.chunk_cubes : tc > 0 ? (uint32_t)tc : 2048u;
        p->threads = o.block_threads > 0 ? o.block_threads : tt > 0 ? tt : 256;
        p->cap_blocks = max_blocks > 0 ? (uint64_t)max_blocks : (uint64_t)max_Q * 1024;
        p->cap_chunks = max_chunks > 0 ? (uint64_t)max_chunks : (uint64_t)max_Q * 256;
        if (p->cap_blocks >= (1ull << 32) || p->cap_chunks >= (1ull << 32))
            st = fail(MG_ERR_UNSUPPORTED, "plan capacities must be below 2^32");
    }
    if (st == MG_OK) {
        const size_t S = g->S, Q = (size_t)max_Q;
        auto r = [](size_t n) { return (n + 255) & ~(size_t)255; };
        // boxes, batch size, results (+ u32 scratch), cube counts, both offset
        // arrays, blocks, chunk map, tile words, tickets
        const size_t tiles = Q;   // at most one tile word pair per box
        const size_t bytes = r(Q * 24) + r(8) + r(16) + r(Q * S * 4) * (p->fp ? 2 : 1) + r(8 * Q) + 2 * r(8 * (Q + 1)) +
                             r(p->cap_blocks * sizeof(Blk)) + 2 * r(p->cap_chunks * 4) + r(16 * tiles) + r(16) +
                             65536;
        st = p->pool.alloc(&g->al, bytes, nullptr);
        if (st == MG_OK) {
            cudaError_t e = cudaStreamSynchronize(nullptr);
            if (e != cudaSuccess) st = cuda_fail(e, "plan pool");
            p->pool.s = nullptr;
        }
        if (st == MG_OK) {
            p->bump = Pool{p->pool.as<unsigned char>(), p->pool.bytes, 0};
            p->boxes = static_cast<int32_t*>(pool_alloc(&p->bump, Q * 24, nullptr));
            p->Qd = static_cast<int64_t*>(pool_alloc(&p->bump, 8, nullptr));
            p->result = pool_alloc(&p->bump, Q * S * 4, nullptr);
            p->io = static_cast<void**>(pool_alloc(&p->bump, 16, nullptr));
            void* io0[2] = {p->boxes, p->result};
            const cudaError_t e = cudaMemcpy(p->io, io0, sizeof(io0), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "plan io slots");
        }
    }
    if (st == MG_OK && p->fp && o.alpha_dtype != MG_F32) st = ensure_alpha16(g, (mg_dtype)o.alpha_dtype, nullptr);
    if (st == MG_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    if (st == MG_OK && o.timing) {
        p->timed = true;
        for (cudaEvent_t& ev : p->ev) {
            const cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess && st == MG_OK) st = cuda_fail(e, "cudaEventCreate");
        }
    }
    if (st == MG_OK) {
        // scratch comes from the plan's pool, so nothing is allocated while capturing
        Alloc al;
        al.a.ctx = &p->bump;
        al.a.alloc = pool_alloc;
        al.a.free = pool_free;
        al.custom = true;
        cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
        if (st == MG_OK) {
            if (!p->fp) st = plan_enqueue<false, float>(p.get(), al, p->cap_stream);
            else if (o.alpha_dtype == MG_F16) st = plan_enqueue<true, __half>(p.get(), al, p->cap_stream);
            else if (o.alpha_dtype == MG_BF16) st = plan_enqueue<true, __nv_bfloat16>(p.get(), al, p->cap_stream);
            else st = plan_enqueue<true, float>(p.get(), al, p->cap_stream);
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(p->cap_stream, &gr);
            p->graph = gr;
            if (st == MG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
        }
        if (st == MG_OK) {
            e = cudaGraphInstantiate(&p->exec, p->graph, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    if (st != MG_OK) return st;
    *out = p.release();
    return MG_OK;
}

MG_API mg_status mg_query_plan_run(mg_query_plan* p, const int32_t* boxes, int64_t Q, void* out, size_t out_capacity,
                                   mg_stream stream) {
    MG_RANGE("mg_query_plan_run");
    using namespace mg;
    if (!p) return fail(MG_ERR_INVALID_ARG, "plan is NULL");
    if (Q < 0 || Q > p->max_Q) return fail(MG_ERR_INVALID_ARG, "Q must be in 0..max_Q");
    if (Q == 0) return MG_OK;
    if (!boxes || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if ((uint64_t)out_capacity < (uint64_t)Q * p->g->S) return fail(MG_ERR_INVALID_ARG, "out_capacity must be >= Q*S");
    if (reinterpret_cast<uintptr_t>(boxes) % 4 || reinterpret_cast<uintptr_t>(out) % 4)
        return fail(MG_ERR_INVALID_ARG, "boxes and out must be 4-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->g->device) MG_CUDA(cudaSetDevice(p->g->device));
    mg_status st = MG_OK;
    // the graph reads the boxes from and accumulates into the caller's buffers
    set_batch_kernel<<<1, 1, 0, s>>>(p->Qd, Q, p->io, boxes, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, s);
    if (e == cudaSuccess) p->ran = true;
    if (e != cudaSuccess) st = cuda_fail(e, "mg_query_plan_run");
    if (prev >= 0 && prev != p->g->device) cudaSetDevice(prev);
    return st;
}

MG_API mg_status mg_query_plan_timing(const mg_query_plan* p, float* plan_ms, float* main_ms) {
    using namespace mg;
    if (!p || !plan_ms || !main_ms) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (!p->timed) return fail(MG_ERR_INVALID_ARG, "plan created without opts->timing");
    if (!p->ran) return fail(MG_ERR_INVALID_ARG, "plan has not run");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->g->device) MG_CUDA(cudaSetDevice(p->g->device));
    cudaError_t e = cudaEventSynchronize(p->ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(plan_ms, p->ev[0], p->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(main_ms, p->ev[1], p->ev[2]);
    if (prev >= 0 && prev != p->g->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "mg_query_plan_timing");
    return MG_OK;
}

MG_API void mg_query_plan_free(mg_query_plan* p) {
    if (!p) return;
    const int dev = p->g->device;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    delete p;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: time the batched query over work-chunk sizes and CTA sizes on the
// caller's own batch and keep the fastest for later calls on this graph.
// ---------------------------------------------------------------------------
extern "C" MG_API mg_status mg_query_autotune(mg_graph* g, const int32_t* boxes, int64_t Q, mg_query_opts* opts,
                                              float* best_ms, mg_stream stream) {
    MG_RANGE("mg_query_autotune");
    using namespace mg;
    if (!g || !opts) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (Q < 1 || !boxes) return fail(MG_ERR_INVALID_ARG, "autotuning needs a non-empty batch");
    if (opts->hist_type != MG_HIST_U32 && opts->hist_type != MG_HIST_F32) return fail(MG_ERR_INVALID_ARG, "bad hist_type");
    if (g->quantised && opts->hist_type == MG_HIST_U32)
        return fail(MG_ERR_UNSUPPORTED, "a quantised graph has no exact weights: use MG_HIST_F32");
    const bool FP = opts->hist_type == MG_HIST_F32;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) MG_CUDA(cudaSetDevice(g->device));
    mg_status st = MG_OK;
    Buf outb;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    int best_c = 0, best_t = 0;
    st = outb.alloc(&g->al, (size_t)Q * g->S * 4, s);
    if (st == MG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(MG_ERR_CUDA, "cudaEventCreate");
    // 512 threads matter when one histogram per CTA fills shared memory
    // (many segments): two CTAs per SM then hold 32 warps instead of 8
    const int chunks[] = {1024, 2048, 4096, 8192, 16384};
    const int threads[] = {128, 256, 512};
    const int nc = (int)(sizeof(chunks) / sizeof(chunks[0])), nt = (int)(sizeof(threads) / sizeof(threads[0]));
    for (int ci = 0; st == MG_OK && ci < nc; ci++) {
        for (int ti = 0; st == MG_OK && ti < nt; ti++) {
            mg_query_opts o = *opts;
            o.layout = MG_LAYOUT_DENSE;
            o.schedule = MG_SCHED_BATCHED;
            o.chunk_cubes = chunks[ci];
            o.block_threads = threads[ti];
            o.timing = 0;
            float ms = 0.f;
            for (int rep = 0; st == MG_OK && rep < 3; rep++) {   // first run warms up
                cudaEventRecord(e0, s);
                st = query_boxes(g, boxes, Q, o, outb.p, (size_t)Q * g->S, nullptr, nullptr, nullptr, s);
                cudaEventRecord(e1, s);
                if (st == MG_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(MG_ERR_CUDA, "autotune sync");
                float t = 0.f;
                if (st == MG_OK) cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms += t;
            }
            if (st == MG_OK && ms < best) {
                best = ms;
                best_c = chunks[ci];
                best_t = threads[ti];
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st == MG_OK) {
        g->tuned_chunk[FP ? 1 : 0] = best_c;
        g->tuned_threads[FP ? 1 : 0] = best_t;
        opts->chunk_cubes = best_c;
        opts->block_threads = best_t;
        if (best_ms) *best_ms = best / 2.f;
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return st;
}

// Record a launch shape found earlier (for example, read from a cache file).
extern "C" MG_API mg_status mg_query_set_tuning(mg_graph* g, int hist_type, int chunk_cubes, int block_threads) {
    using namespace mg;
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (hist_type != MG_HIST_U32 && hist_type != MG_HIST_F32) return fail(MG_ERR_INVALID_ARG, "bad hist_type");
    if (chunk_cubes < 0 || (block_threads && block_threads != 128 && block_threads != 256 && block_threads != 512))
        return fail(MG_ERR_INVALID_ARG, "bad launch shape");
    g->tuned_chunk[hist_type] = chunk_cubes;
    g->tuned_threads[hist_type] = block_threads;
    return MG_OK;
}
