// bsi_geometry.h -- index arithmetic shared by the kernels and the host.
//
// Every global or shared-memory range a kernel touches is computed by one of
// these functions.  They compile for the device (kernels) and for the host
// (launch set-up and bsi_selfcheck_ranges, which walks every unit of a launch
// on the CPU and checks each range against its buffer before anything runs).
//
// Work decomposition (Sec. 2.1.1: a tile is one control cell of dx*dy*dz
// voxels, and all voxels of a tile share the same 4x4x4 control points):
//  * a warp owns a UNIT: a strip of up to 29 x-neighbouring tiles of one
//    tile-row (jy) and one tile-plane (kz) -- forward -- or of a chunk of
//    tile-planes -- adjoint.  Lane l holds one column of control points, so a
//    warp holds 32 columns and completes 32 - 3 = 29 tiles (forward) or the
//    full sums of 29 columns (adjoint); the 3 extra lanes are the halo of the
//    4-wide neighbourhood.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define BSI_HD __host__ __device__ __forceinline__
#else
#define BSI_HD inline
#endif

namespace bsi {

constexpr int kLanes = 32;
constexpr int kHalo = 3;                       // neighbourhood width 4 = 1 + kHalo
constexpr int kGroupCells = kLanes - kHalo;    // tiles (forward) or columns (adjoint) per warp
constexpr int kMaxSpacing = 64;
constexpr int kMaxSpecializedDx = 8;           // x-spacings with a compile-time inner loop
constexpr int kMaxBatch = 64;                  // instances per launch (kernel parameters)

// One volume as the kernels see it.  Filled on the host from bsi_geom.
struct InstDesc {
    int X, Y, Z;
    int dx, dy, dz;
    int nx, ny, nz;      // stored control grid
    int ncx, ncy, ncz;   // tiles per axis (0 for an empty volume)
    int nxg;             // x-groups: ceil(ncx/29) forward, ceil(nx/29) adjoint
    int nzc;             // adjoint: tile-plane chunks
    int zchunk;          // adjoint: tile-planes per chunk
    int gcells;          // forward: tiles per warp strip (<= 29; see fwd_strip_tiles)
    int warps_req;       // requested warps per CTA from the tile-config table (0: automatic)
    int tma_rows;        // adjoint tensor-copy path: rows per block (tma_block_rows), else 0
    int jrows;           // adjoint: tile-rows per unit (1, or 2 on the tensor-copy path)
    int ncyu;            // adjoint: unit rows, ceil(ncy / jrows)
    long long units;        // units of this instance
    long long unit_begin;   // first global unit index of this instance in its launch
    long long point_begin;  // adjoint reduce: first global grid point of this instance
    long long part_off;     // adjoint: float offset of this instance's partials in the workspace
    const float* phi;
    void* field;
    const float* grad;
    float* dphi;
    // resampling of a floating image by the field (bsi_resample_*)
    const float* image;     // floating image [fZ][fY][fX]
    const float* gwarp;     // gradient mode: dL/dwarped [Z][Y][X]
    int fX, fY, fZ;
    int rpad;
};

template <int MAXB>
struct Batch {
    int n;
    int buf_bytes;          // bytes of one staging row slot (stage_buf_bytes of the largest dx)
    int warps_req;          // requested warps per CTA (0: as many as shared memory allows, <= 8)
    int stages;             // adjoint tensor-copy path: ring stages per warp (else 0)
    long long total_units;
    long long total_points;
    InstDesc inst[MAXB];
};

// Index of instance i in a launch's descriptor array: the constant 0 when the
// launch holds one instance (MAXB == 1), so that the descriptor's fields are
// constant-bank operands rather than loads indexed by a register.
template <int MAXB>
BSI_HD int inst_index(int i) { return MAXB == 1 ? 0 : i; }

BSI_HD long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
BSI_HD int imin(int a, int b) { return a < b ? a : b; }
BSI_HD int imax(int a, int b) { return a > b ? a : b; }

// Offset of the 4*d weights of spacing d in the weight table: sum_{e<d} 4e.
BSI_HD constexpr int weight_base(int d) { return 2 * d * (d - 1); }
constexpr int kWeightCount = weight_base(kMaxSpacing + 1);

// Element (float or bf16) offset of voxel (x, y, z) channel 0 in a field.
BSI_HD long long field_elem(const InstDesc& d, int z, int y, int x) {
    return (((long long)z * d.Y + y) * d.X + x) * 3;
}

// Float offset of stored control point (gx, gy, gz) channel 0.
BSI_HD long long phi_elem(const InstDesc& d, int gz, int gy, int gx) {
    return (((long long)gz * d.ny + gy) * d.nx + gx) * 3;
}

// Unit taken by slot (cta, warp) in round r of a persistent launch of `ctas`
// CTAs x `wpc` warps over `total` units, or -1 when the slot has none.  Full
// rounds are CTA-major (the warps of a CTA take neighbouring units, which share
// control points in L1 and, in a batch, a kernel specialisation); the last,
// partial round is dealt warp-major across the CTAs (spread_tail) so that every
// SM gets an even share of it -- worth it for the adjoint's few long units,
// not for the forward's many short ones.
BSI_HD long long slot_unit(long long r, int cta, int warp, int ctas, int wpc, long long total,
                           bool spread_tail = true) {
    const long long W = (long long)ctas * wpc;
    const long long base = r * W;
    if (base >= total) return -1;
    if (total - base >= W || !spread_tail) {
        const long long u = base + (long long)cta * wpc + warp;
        return u < total ? u : -1;
    }
    const long long p = (long long)warp * ctas + cta;
    return p < total - base ? base + p : -1;
}

// ---------------------------------------------------------------- forward

struct FwdUnit {
    int kz, jy, xg;
    int cell0;   // first tile of the strip; lane l holds grid column cell0 + l
    int ncell;   // tiles the warp outputs (<= 29)
    int x0;      // first voxel of the strip
    int nvox;    // voxels per row of the strip
};

// Tiles per forward strip.  When a row of the field is a multiple of 16 bytes
// (X % 4 == 0 for FP32 output, X % 8 == 0 for BF16), a strip of g tiles whose
// byte width 3 g dx ES is a multiple of 16 starts every row segment on a
// 16-byte boundary, so each row leaves as one aligned bulk copy with no
// unaligned head or tail: the largest such g <= 29 (FP32: 28 or 29; BF16 at
// even dx: 28 or 29).  BF16 at odd dx would need g = 24, whose idle lanes cost
// more than the unaligned ends save (512 x 512 x 300 at spacing 5: 0.172 ->
// 0.181 ms): 29, as when rows are unaligned anyway.  (One channel of 4 or 2
// bytes gives the same conditions.)
BSI_HD int fwd_strip_tiles(int X, int dx, bool bf16) {
    const int q = bf16 ? 8 : 4;   // g dx must be a multiple of q
    if (X % q != 0 || (bf16 && dx % 2 != 0)) return kGroupCells;
    for (int g = kGroupCells; g > 1; --g)
        if ((g * dx) % q == 0) return g;
    return kGroupCells;
}

BSI_HD FwdUnit fwd_unit(const InstDesc& d, long long ul) {
    FwdUnit u;
    if (d.units <= 0x7fffffffLL) {   // 32-bit division (64-bit division is a long sequence)
        const unsigned t = (unsigned)ul / (unsigned)d.nxg;
        u.xg = (int)((unsigned)ul - t * (unsigned)d.nxg);
        u.jy = (int)(t % (unsigned)d.ncy);
        u.kz = (int)(t / (unsigned)d.ncy);
    } else {
        u.xg = (int)(ul % d.nxg);
        const long long t = ul / d.nxg;
        u.jy = (int)(t % d.ncy);
        u.kz = (int)(t / d.ncy);
    }
    u.cell0 = u.xg * d.gcells;
    u.ncell = imin(d.gcells, d.ncx - u.cell0);
    u.x0 = u.cell0 * d.dx;
    u.nvox = imin(u.ncell * d.dx, d.X - u.x0);
    return u;
}

// ---------------------------------------------------------------- adjoint

struct AdjUnit {
    int zc, jy, xg;   // jy: the unit's first tile-row (it takes jrows of them)
    int col0;    // first complete column; lane l holds tile / column col0 - 3 + l
    int xs;      // first voxel read by the warp
    int nvox;    // voxels per row read by the warp
    int kz0, kz1;
};

BSI_HD AdjUnit adj_unit(const InstDesc& d, long long ul) {
    AdjUnit u;
    u.xg = (int)(ul % d.nxg);
    const long long t = ul / d.nxg;
    u.jy = (int)(t % d.ncyu) * d.jrows;
    u.zc = (int)(t / d.ncyu);
    u.col0 = u.xg * kGroupCells;
    const int c_lo = imax(0, u.col0 - kHalo);
    const int c_hi = imin(d.ncx, u.col0 + kGroupCells);
    u.xs = c_lo * d.dx;
    u.nvox = c_hi > c_lo ? imin(d.X, c_hi * d.dx) - u.xs : 0;
    u.kz0 = u.zc * d.zchunk;
    u.kz1 = imin(d.ncz, u.kz0 + d.zchunk);
    return u;
}

// Floats of partial sums one adjoint unit writes: (zchunk + 3) planes x
// (jrows + 3) grid rows x 29 columns x 3 channels.
BSI_HD long long adj_unit_floats(const InstDesc& d) {
    return (long long)(d.zchunk + kHalo) * (d.jrows + kHalo) * kGroupCells * 3;
}

// Partial sum of a unit: grid plane pz of its window, grid row m (0 .. jrows + 2,
// from its first tile-row), column j.
BSI_HD long long part_elem(const InstDesc& d, long long ul, int pz, int m, int j) {
    return d.part_off + ul * adj_unit_floats(d) + (((long long)pz * (d.jrows + kHalo) + m) * kGroupCells + j) * 3;
}

// Staging buffer bytes for a largest x-spacing dxmax: one row segment of up to
// 32 tiles x dxmax voxels x 3 FP32 channels, plus up to 15 bytes of alignment
// shift on each side (the adjoint's bulk loads cover the 16-byte-aligned
// superset of a row segment).
BSI_HD int stage_buf_bytes(int dxmax) {
    const int b = 32 + kLanes * dxmax * 3 * 4;
    return (b + 15) & ~15;
}

constexpr int kStoreStages = 3;   // forward: ring of staging buffers per warp (bulk stores in flight)
constexpr int kLoadStages = 4;    // adjoint: ring of staging buffers per warp (bulk loads in flight)

// Shared memory of one warp: forward -- the store ring; adjoint -- one 16-byte
// mbarrier slot per stage, then the load ring.
BSI_HD int fwd_warp_smem(int buf_bytes) { return kStoreStages * buf_bytes; }
BSI_HD int adj_warp_smem(int buf_bytes) { return kLoadStages * (16 + buf_bytes); }

// Forward on the tensor-store path (one volume, three channels): when every row
// of the field is a multiple of 16 bytes and every strip starts on a 16-byte
// boundary, a warp stages rb rows of its strip (a block) and writes the block
// with one tensor store instead of one bulk copy per row.  The box is the
// strip's row as 8-byte elements (at most 256) x rb rows x 1 plane; rb divides
// the y-spacing, so that a block never reaches into the next tile-row, and the
// warp's kStoreStages blocks (128-byte aligned, plus a 128-byte slot the halo
// lanes stage into) fit 1/16 of an SM's shared memory (two 8-warp CTAs).
constexpr int kFwdTmaWarpBudget = 14 * 1024;
constexpr int kBf16OddStripTiles = 24;   // BF16 strips at odd x-spacings on that path: 6 g dx % 16 == 0
BSI_HD int pad128(int b) { return (b + 127) & ~127; }
BSI_HD int fwd_tma_row_bytes(int gcells, int dx, bool bf16, int c = 3) { return gcells * dx * c * (bf16 ? 2 : 4); }
BSI_HD int fwd_tma_warp_smem(int blk_bytes) { return kStoreStages * blk_bytes + 128; }

// Rows per block of the tensor-store path, or 0 where it does not apply
// (rows or strips off 16-byte boundaries, boxes wider than 256 elements, no
// divisor of dy >= 2 whose blocks fit, or FP32 output at x-spacings >= 5).
// Measured on 512^3: FP32 at spacing 3 0.389 -> 0.352 ms and at 4 0.269 ->
// 0.250 ms (bound by per-row work); BF16 at 4, 6, 8 14-16% faster; FP32 at 6,
// already at the write roofline, 0.231 -> 0.246 ms (so not taken).
BSI_HD int fwd_tma_rows(int X, int dx, int dy, int gcells, bool bf16, int c = 3) {
    const int rowb = fwd_tma_row_bytes(gcells, dx, bf16, c);
    if (dx < 1 || dx > (bf16 ? kMaxSpecializedDx : 4) || (c * X * (bf16 ? 2 : 4)) % 16 != 0 || rowb % 16 != 0 ||
        rowb / 8 > 256)
        return 0;
    for (int rb = dy; rb >= 2; --rb)
        if (dy % rb == 0 && fwd_tma_warp_smem(pad128(rb * rowb)) <= kFwdTmaWarpBudget) return rb;
    return 0;
}

// ---------------------------------------------------------------- adjoint, tensor-copy path
//
// When the voxel gradient's rows are 16-byte multiples (X % 4 == 0) and
// dx <= 8, the adjoint fetches its input with TMA tensor copies from a 3-D
// view of the gradient as 8-byte elements (pairs of floats): (3X/2, Y, Z).
// One ring stage holds a BLOCK: rb consecutive rows of a voxel plane of the
// unit's tile-row, 32 tiles wide (rb divides dy, so a plane is dy / rb blocks).
// A box row is one contiguous run of a gradient row (<= 256 elements per box
// dimension): one box of 48 dx + 2 elements for dx <= 5, else two boxes of
// 24 dx + 2 elements, lanes 0..15 reading the first and 16..31 the second.
// The first box starts at the 16-byte group holding the unit's first float,
// which may lie before the array: elements outside it arrive as zeros.
BSI_HD int tma_boxes(int dx) { return dx <= 5 ? 1 : 2; }
BSI_HD int tma_box_width(int dx) { return tma_boxes(dx) == 1 ? 48 * dx + 2 : 24 * dx + 2; }
// Shared bytes of one box of rb rows, padded to the 128 bytes a tensor copy's
// destination is aligned to.
BSI_HD int tma_box_bytes(int dx, int rb) { return (8 * tma_box_width(dx) * rb + 127) & ~127; }
BSI_HD int tma_block_bytes(int dx, int rb) { return tma_boxes(dx) * tma_box_bytes(dx, rb); }

constexpr int kTmaMaxRows = 8;                   // rows per block
constexpr int kTmaBlockTarget = 14 * 1024;       // largest block that still leaves room for 2 stages x 8 warps
constexpr int kTmaMinStages = 2;
constexpr int kTmaMaxStages = 4;
constexpr int kTmaMaxWarps = 12;                 // register budget: 12 warps x 32 x 170 <= 65536
constexpr int kTmaMaxWarps2 = 11;                // two tile-rows per unit: 11 warps x 32 x 186
constexpr int kTmaSmemBudget = 227 * 1024;       // one CTA per SM takes all of its shared memory

// Rows per block for spacing (dx, dy): the largest divisor of dy up to
// kTmaMaxRows whose block fits kTmaBlockTarget (1 always does).
BSI_HD int tma_block_rows(int dx, int dy) {
    for (int rb = imin(dy, kTmaMaxRows); rb > 1; --rb)
        if (dy % rb == 0 && tma_block_bytes(dx, rb) <= kTmaBlockTarget) return rb;
    return 1;
}
// Shared memory of one warp: 128 bytes of mbarriers, then the ring of stages.
BSI_HD int tma_warp_smem(int stage_bytes, int stages) { return 128 + stages * stage_bytes; }
// Default ring depth for a stage size, 2 or 3: 3 where it still fits beside
// 12 warps (measured: a 4th stage slowed small blocks down; 3 beat 2 where
// both fit), and also where two stages fall short of 12 warps anyway while
// three keep at least 7.  Measured on the 512 x 512 x 300 volume at spacing 5
// (9.7 KB stages: 11 warps x 2 stages or 7 warps x 3): equal alone, 11 us
// faster right after a forward, whose field is still leaving L2 -- the deeper
// ring rides out the longer load latency.  Where two stages reach 12 warps
// (512^3 at spacing (4,5,6)) or three would leave 6 (spacing 8), fewer warps
// cost 12-25% and the ring stays at 2.
constexpr int kTmaMinDeepWarps = 7;
BSI_HD int tma_default_stages(int stage_bytes) {
    const int w2 = (kTmaSmemBudget - 128) / tma_warp_smem(stage_bytes, 2);
    const int w3 = (kTmaSmemBudget - 128) / tma_warp_smem(stage_bytes, 3);
    return (w3 >= kTmaMaxWarps || (w2 < kTmaMaxWarps && w3 >= kTmaMinDeepWarps)) ? 3 : 2;
}

// Float index (x * 3 + channel) of the unit's first float and its 16-byte group.
BSI_HD int tma_first_float(const AdjUnit& u, int dx) { return (u.col0 - kHalo) * 3 * dx; }
BSI_HD int tma_group_of(int f) { return f >= 0 ? f / 4 : -((-f + 3) / 4); }   // floor(f / 4)

// ---------------------------------------------------------------- non-integer spacing

// One volume with spacing num/den and lattice shift off/den per axis (x, y, z).
struct RatDesc {
    int X, Y, Z;
    int num[3], den[3], off[3];
    int nx, ny, nz;
    const float* phi;
    float* field;
};

// Stored grid points along one axis: floor(((N - 1) den + off) / num) + 4.
BSI_HD long long rational_dim(long long N, int num, int den, int off) {
    return N > 0 ? ((N - 1) * den + off) / num + 4 : 4;
}

constexpr int kMaxWarpsPerCta = 8;
constexpr int kAdjWarpsMax = 4;   // adjoint partials kernel: 4-warp CTAs (register budget)
constexpr int kSmemBudget = 200 * 1024;   // dynamic shared memory per CTA we allow

// Warps per CTA such that the warps' shared memory fits the budget, at most
// `req` when a tile config asks for fewer (req = 0: no request).
BSI_HD int warps_per_cta(int warp_smem, int req = 0) {
    int w = kSmemBudget / warp_smem;
    if (req > 0 && req < w) w = req;
    return w < 1 ? 1 : (w > kMaxWarpsPerCta ? kMaxWarpsPerCta : w);
}

}  // namespace bsi
