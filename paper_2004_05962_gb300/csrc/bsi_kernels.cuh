// bsi_kernels.cuh -- sm_103a kernels for cubic B-spline interpolation (BSI).
//
// Forward (Eq. 1, Sec. 2.1), evaluated by sum factorisation: for a tile the
// 4x4x4 neighbourhood is contracted along z, then y, then x, so a voxel costs
// 12 FMAs (4 taps x 3 channels) plus the z and y stages shared by the tiles of
// a warp, instead of the 255 (direct) or 126 (trilinear rewrite) operations
// per channel counted in App. B.
//
// Each warp owns a strip of tiles (see bsi_geometry.h).  Lane l keeps the 4x4
// column of control displacements at grid column cell0 + l in registers (the
// register reuse of Sec. 3.2.2, one column per lane instead of one 4x4x4 cube
// per thread), contracts it along z and y, and takes the three x-neighbour
// columns from lanes l+1..l+3 with shuffles.  Each output row segment is
// staged in shared memory and leaves the SM as one bulk copy (TMA) of its
// 16-byte-aligned body plus a few plain stores for the unaligned ends; a ring
// of kStoreStages buffers per warp keeps copies in flight while the next rows
// are computed.  The paper found its one-thread-per-tile stores uncoalesced
// and bandwidth-limiting (Sec. 5.2.1); here every row leaves as contiguous
// 16-byte-aligned bulk transfers.
//
// Adjoint (transpose of Eq. 1): the same strip walked in the opposite
// direction.  Rows of the voxel gradient arrive by bulk copy into a ring of
// kLoadStages buffers per warp (mbarrier completion, issued kLoadStages rows
// ahead); each lane applies the x-transpose to its tile, a column collects
// the four tiles that touch it with shuffles, and y and z are accumulated in
// registers into per-unit partial sums that a second kernel reduces in a
// fixed order (no atomics, bitwise reproducible).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsi_async.cuh"
#include "bsi_geometry.h"
#include "bsi_weights.cuh"

namespace bsi {

constexpr unsigned kFull = 0xffffffffu;

// Kernel error bits (range bits only in checked builds; kErrTimeout always).
enum : unsigned {
    kErrPhiRead = 1u,
    kErrFieldWrite = 2u,
    kErrStage = 4u,
    kErrGradRead = 8u,
    kErrPartWrite = 16u,
    kErrPartRead = 32u,
    kErrDphiWrite = 64u,
    kErrTimeout = 128u,
};

#ifdef BSI_CHECKED
#define BSI_GUARD(cond, bit, err)        \
    if (!(cond)) {                       \
        atomicOr((err), (bit));          \
    } else
#else
#define BSI_GUARD(cond, bit, err)
#endif

__device__ __forceinline__ uintptr_t floor16(uintptr_t a) { return a & ~(uintptr_t)15; }
__device__ __forceinline__ uintptr_t ceil16(uintptr_t a) { return (a + 15) & ~(uintptr_t)15; }

// Stores one voxel's C channels at shared address s (FP32, or BF16 rounded to
// nearest even).
template <bool BF16, int C>
__device__ __forceinline__ void put_voxel(uint32_t s, const float (&v)[C]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (BF16) sts_b16(s + 2 * c, __bfloat16_as_ushort(__float2bfloat16_rn(v[c])));
        else sts_f32(s + 4 * c, v[c]);
    }
}

// ------------------------------------------------------------------ forward

// Writes one staged row segment [g, g + nbytes) (staged at sb, congruent to g
// mod 16; shift = g mod 16): lane 0 hands the 16-byte-aligned body to the
// bulk-copy engine, commits one bulk group and then waits until at most
// kStoreStages - 1 groups still read shared memory, which frees the ring
// buffer the warp writes next; lanes store the < 16-byte head and tail.
template <int ES>
__device__ __forceinline__ void store_row(const unsigned char* sb, unsigned char* g, int shift, int nbytes,
                                          int lane) {
    if (shift == 0 && (nbytes & 15) == 0) {  // aligned segment (warp-uniform): one bulk copy, no ends
        if (lane == 0) {
            bulk_store(g, sb, (uint32_t)nbytes);
            bulk_commit();
            bulk_wait_read<kStoreStages - 1>();
        }
        return;
    }
    int head = (16 - shift) & 15;
    head = head < nbytes ? head : nbytes;
    const int body = (nbytes - head) & ~15;
    if (lane == 0) {
        if (body > 0) bulk_store(g + head, sb + head, (uint32_t)body);
        bulk_commit();
        bulk_wait_read<kStoreStages - 1>();
    }
    const int nh = head / ES, nt = (nbytes - head - body) / ES;
    const int off = lane < nh ? lane * ES : head + body + (lane - nh) * ES;
    if (lane < nh + nt) {
        if (ES == 4) *reinterpret_cast<uint32_t*>(g + off) = *reinterpret_cast<const uint32_t*>(sb + off);
        else *reinterpret_cast<uint16_t*>(g + off) = *reinterpret_cast<const uint16_t*>(sb + off);
    }
}

// v = w0 p0 + w1 p1 + w2 p2 + w3 p3 per channel, as a multiply and three fused
// multiply-adds in that order.  PACK takes channels 0 and 1 through the packed
// FP32x2 multiply and FMA of sm_100-class GPUs: per channel the same
// operations in the same order, so the results equal the scalar form's bit
// for bit, in about two thirds of the instructions.
template <int C, bool PACK>
__device__ __forceinline__ void combine4(float (&v)[C], float w0, float w1, float w2, float w3, const float (&p0)[C],
                                         const float (&p1)[C], const float (&p2)[C], const float (&p3)[C]) {
    if constexpr (C == 3 && PACK) {
        float2 a = __fmul2_rn(make_float2(w0, w0), make_float2(p0[0], p0[1]));
        a = __ffma2_rn(make_float2(w1, w1), make_float2(p1[0], p1[1]), a);
        a = __ffma2_rn(make_float2(w2, w2), make_float2(p2[0], p2[1]), a);
        a = __ffma2_rn(make_float2(w3, w3), make_float2(p3[0], p3[1]), a);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = fmaf(w3, p3[2], fmaf(w2, p2[2], fmaf(w1, p1[2], w0 * p0[2])));
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = fmaf(w3, p3[c], fmaf(w2, p2[c], fmaf(w1, p1[c], w0 * p0[c])));
    }
}

// Whether the forward's z, y and x stages use the packed form of combine4:
// where a row's instructions bound the kernel -- BF16 output, x-spacings <= 3
// (measured 8% and 4% faster) -- and not for FP32 output at larger spacings,
// which is bound by its stores and measured up to 8% slower with it.
template <int DX, bool BF16>
__host__ __device__ constexpr bool fwd_packed() {
    return BF16 || (DX > 0 && DX <= 3);
}

// Two values rounded to BF16 (nearest even) in one 32-bit word, lo at the
// lower address.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    uint32_t w;
    memcpy(&w, &h, sizeof(w));
    return w;
}

// Stores the N values of a lane's tile as BF16 (nearest even) from shared byte
// address s (2-byte aligned), two values per 32-bit word, each pair converted
// by one packed instruction; 8- or 16-byte stores where the start allows.  A
// run starting 2 bytes past a word boundary stores its first value alone and
// then the pairs shifted by one value (each word a byte permute of two
// neighbouring converted pairs).  One 16-bit store per value, at the lane
// stride of 6 DX bytes, meets up to 4-way bank conflicts (x-spacing 8: 0.35 ->
// 0.19 ms for 512^3).  Odd N (odd x-spacings): neighbouring lanes alternate
// between the two alignments, so each lane picks its permutation at run time;
// on the per-row store path that measured 1.5% slower than 16-bit stores and
// is not used there, on the tensor-store path 7% faster (512 x 512 x 300 at
// spacing 5: 0.146 -> 0.136 ms).
template <int N>
__device__ __forceinline__ void sts_bf16_run(uint32_t s, const float (&v)[N]) {
    if constexpr (N % 2 == 0) {
        uint32_t w[N / 2];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) w[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
        // runs 2N bytes apart: every lane of the warp takes the same branch
        if ((s & 2u) == 0) {
            if (N % 8 == 0 && (s & 15u) == 0) {
#pragma unroll
                for (int j = 0; j < N / 2; j += 4) sts_v4_b32(s + 4 * j, w[j], w[j + 1], w[j + 2], w[j + 3]);
            } else if (N % 4 == 0 && (s & 7u) == 0) {
#pragma unroll
                for (int j = 0; j < N / 2; j += 2) sts_v2_b32(s + 4 * j, w[j], w[j + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < N / 2; ++j) sts_b32(s + 4 * j, w[j]);
            }
        } else {
            sts_b16(s, (unsigned short)(w[0] & 0xffffu));
#pragma unroll
            for (int j = 0; j + 1 < N / 2; ++j) sts_b32(s + 2 + 4 * j, __byte_perm(w[j], w[j + 1], 0x5432));
            sts_b16(s + 2 * (N - 1), (unsigned short)(w[N / 2 - 1] >> 16));
        }
    } else {
        // (N + 1) / 2 pairs, the last one padded with a zero
        uint32_t w[N / 2 + 1];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) w[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
        w[N / 2] = pack_bf16x2(v[N - 1], 0.f);
        // word-aligned start: pairs (0,1), (2,3), ... then the last value alone;
        // 2 bytes past: the first value alone, then pairs (1,2), (3,4), ...
        const uint32_t odd = (s >> 1) & 1u;
        const uint32_t sel = odd ? 0x5432u : 0x3210u;
#pragma unroll
        for (int j = 0; j < N / 2; ++j) sts_b32(s + 2 * odd + 4 * j, __byte_perm(w[j], w[j + 1], sel));
        sts_b16(odd ? s : s + 2 * (N - 1), (unsigned short)((odd ? w[0] : w[N / 2]) & 0xffffu));
    }
}

// x-stage of one voxel of a tile: out = sum_l B_l(r/dx) p_l, per channel (C of
// them: 3 for the displacement field, 1 for scalar interpolation), staged at
// shared address s.
template <bool BF16, int C, bool PK = false>
__device__ __forceinline__ void emit_voxel(uint32_t s, int wo, const float (&p0)[C], const float (&p1)[C],
                                           const float (&p2)[C], const float (&p3)[C]) {
    const float w0 = c_lut.w[wo], w1 = c_lut.w[wo + 1], w2 = c_lut.w[wo + 2], w3 = c_lut.w[wo + 3];
    float v[C];
    combine4<C, PK>(v, w0, w1, w2, w3, p0, p1, p2, p3);
    put_voxel<BF16, C>(s, v);
}

// Shared-memory vector width (floats) for staging the C DX FP32 values of one
// lane's tile: a lane's tile starts 4 C DX bytes after its neighbour's, so with
// DX a multiple of 4 (2) and an aligned row start it can move 16 (8) bytes per
// access -- 4 (2) times fewer LDS/STS, and for DX = 4, 6, 8 fewer bank
// conflicts than the 4 C DX-byte scalar stride (C = 1 or 3, odd).
template <int DX>
__host__ __device__ constexpr int tile_vec() {
    return DX <= 0 ? 1 : (DX % 4 == 0 ? 4 : (DX % 2 == 0 ? 2 : 1));
}

// x-stage of a whole tile of DX voxels staged from shared address sv: FP32
// with VW-float stores (sv aligned to 4 VW bytes), BF16 through sts_bf16_run
// when the tile holds an even number of values or ODD_WORDS is set (the
// tensor-store path), else one value at a time.
template <int DX, int VW, bool BF16, int C, bool PK = fwd_packed<DX, BF16>(), bool ODD_WORDS = false>
__device__ __forceinline__ void emit_tile(uint32_t sv, const float (&p0)[C], const float (&p1)[C],
                                          const float (&p2)[C], const float (&p3)[C]) {
    constexpr bool kWords = BF16 && ((C * DX) % 2 == 0 || ODD_WORDS);
    if (!kWords && VW == 1) {
#pragma unroll
        for (int r = 0; r < DX; ++r)
            emit_voxel<BF16, C, PK>(sv + C * (BF16 ? 2 : 4) * r, weight_base(DX) + 4 * r, p0, p1, p2, p3);
    } else {
        float v[C * DX];
#pragma unroll
        for (int r = 0; r < DX; ++r) {
            const int wo = weight_base(DX) + 4 * r;
            float t[C];
            combine4<C, PK>(t, c_lut.w[wo], c_lut.w[wo + 1], c_lut.w[wo + 2], c_lut.w[wo + 3], p0, p1, p2, p3);
#pragma unroll
            for (int c = 0; c < C; ++c) v[C * r + c] = t[c];
        }
        if constexpr (kWords) {
            sts_bf16_run<C * DX>(sv, v);
        } else {
#pragma unroll
            for (int i = 0; i < C * DX / VW; ++i) {
                if (VW == 4) sts_v4_f32(sv + 16 * i, v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                else sts_v2_f32(sv + 8 * i, v[2 * i], v[2 * i + 1]);
            }
        }
    }
}

// One forward unit: tile-plane kz, tile-row jy, x-group xg.  DX > 0 is a
// compile-time x-spacing (unrolled inner loop, weights as constant operands);
// DX == 0 reads the spacing at run time.  ring is the warp's next staging
// buffer in its store ring (0 .. kStoreStages - 1).  C channels per control
// point and voxel: 3 (the displacement field) or 1 (scalar interpolation,
// layouts [nz][ny][nx] and [Z][Y][X]).
template <int DX, bool BF16, int C = 3, bool PACK_ALL = false>
__device__ __forceinline__ void forward_unit(const InstDesc& d, long long ul, unsigned char* stage,
                                             int buf_bytes, int lane, int& ring, unsigned* err) {
    static_assert(C == 1 || C == 3, "one (scalar) or three (displacement) channels");
    constexpr int ES = BF16 ? 2 : 4;
    constexpr bool PK = PACK_ALL || fwd_packed<DX, BF16>();
    const int dx = DX > 0 ? DX : d.dx;
    const FwdUnit u = fwd_unit(d, ul);
    const int col = u.cell0 + lane;

    // 4 (z) x 4 (y) neighbourhood column of control points, C channels.
    float ph[4][4][C];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (C == 3) {
                float a = 0.f, b = 0.f, c = 0.f;
                if (col < d.nx) {
                    const long long e = phi_elem(d, u.kz + n, u.jy + m, col);
                    BSI_GUARD(e >= 0 && e + 3 <= 3LL * d.nx * d.ny * d.nz, kErrPhiRead, err) {
                        const float* p = d.phi + e;
                        a = __ldg(p);
                        b = __ldg(p + 1);
                        c = __ldg(p + 2);
                    }
                }
                ph[n][m][0] = a;
                ph[n][m][C > 1 ? 1 : 0] = b;
                ph[n][m][C > 2 ? 2 : 0] = c;
            } else {
                float a = 0.f;
                if (col < d.nx) {
                    const long long e = ((long long)(u.kz + n) * d.ny + (u.jy + m)) * d.nx + col;
                    BSI_GUARD(e >= 0 && e < (long long)d.nx * d.ny * d.nz, kErrPhiRead, err) { a = __ldg(d.phi + e); }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) ph[n][m][c] = a;
            }
        }

    const int z0 = u.kz * d.dz, zn = imin(d.dz, d.Z - z0);
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const int wzb = weight_base(d.dz), wyb = weight_base(d.dy), wxb = weight_base(dx);
    const int xl = lane * dx;                 // first strip voxel of this lane's tile
    // voxels of this lane's tile inside the strip (0 for the halo lanes)
    const int rn = lane < u.ncell ? imin(dx, u.nvox - xl) : 0;
    const int nbytes = u.nvox * C * ES;
    const long long row_pitch = (long long)C * d.X * ES;   // bytes from row y to row y + 1
    const long long plane_pitch = row_pitch * d.Y;       // bytes from plane z to plane z + 1
    unsigned char* gplane =
        static_cast<unsigned char*>(d.field) + ((((long long)z0 * d.Y + y0) * d.X + u.x0) * C) * ES;   // field_elem for C
    // every row of the unit starts on a 16-byte boundary (x0 is a multiple of DX)
    const bool direct = C == 1 && (reinterpret_cast<uintptr_t>(d.field) & 15) == 0 && (d.X & 3) == 0;

    for (int rz = 0; rz < zn; ++rz, gplane += plane_pitch) {
        const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
        const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
        float pz[4][C];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            combine4<C, PK>(pz[m], a0, a1, a2, a3, ph[0][m], ph[1][m], ph[2][m], ph[3][m]);

        unsigned char* g = gplane;
        for (int ry = 0; ry < yn; ++ry, g += row_pitch) {
            const float b0 = c_lut.w[wyb + 4 * ry], b1 = c_lut.w[wyb + 4 * ry + 1];
            const float b2 = c_lut.w[wyb + 4 * ry + 2], b3 = c_lut.w[wyb + 4 * ry + 3];
            float p0[C], p1[C], p2[C], p3[C];
            combine4<C, PK>(p0, b0, b1, b2, b3, pz[0], pz[1], pz[2], pz[3]);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                p1[c] = __shfl_down_sync(kFull, p0[c], 1);
                p2[c] = __shfl_down_sync(kFull, p0[c], 2);
                p3[c] = __shfl_down_sync(kFull, p0[c], 3);
            }

            if constexpr (C == 1 && !BF16 && DX == 4) {
                if (direct) {
                    // one-channel FP32 rows on 16-byte boundaries at x-spacing 4: a lane's
                    // tile is one 16-byte vector, so the warp's stores of its tiles are
                    // contiguous -- no staging, no bulk copy (0.103 -> 0.074 ms for a 4x
                    // zoom to 512 x 512 x 300; at spacing 8 two vectors per lane leave
                    // each store instruction half-sector gaps and the bulk copy wins)
                    BSI_GUARD(rn == 0 || (g - static_cast<unsigned char*>(d.field)) / 4 + xl + rn <=
                                             (long long)d.X * d.Y * d.Z, kErrFieldWrite, err) {
                        if (rn > 0) {
                            float v[DX];
#pragma unroll
                            for (int r = 0; r < DX; ++r) {
                                const int wo = weight_base(DX) + 4 * r;
                                const float w0 = c_lut.w[wo], w1 = c_lut.w[wo + 1], w2 = c_lut.w[wo + 2],
                                            w3 = c_lut.w[wo + 3];
                                v[r] = fmaf(w3, p3[0], fmaf(w2, p2[0], fmaf(w1, p1[0], w0 * p0[0])));
                            }
                            float4* o = reinterpret_cast<float4*>(g + 4 * xl);
#pragma unroll
                            for (int i = 0; i < DX / 4; ++i)
                                if (4 * i < rn) __stcs(o + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
                        }
                    }
                    continue;
                }
            }
            const int shift = (int)(reinterpret_cast<uintptr_t>(g) & 15);
            unsigned char* sb = stage + ring * buf_bytes + shift;
            ring = ring == kStoreStages - 1 ? 0 : ring + 1;
            // (the ring buffer is free: store_row of the previous row waited for it)
            BSI_GUARD(shift + (DX > 0 ? C * ES * kLanes * DX : nbytes) <= buf_bytes, kErrStage, err) {
                // shared address of this lane's first voxel
                const uint32_t sv = smem_u32(sb) + (uint32_t)(C * ES * xl);
                if (DX > 0) {
                    // every lane stages all DX voxels of its tile, unpredicated: a cut or
                    // halo tile lands past the row end, inside the buffer (lane 31 ends at
                    // 32 DX voxels), and only [shift, shift + nbytes) is copied out
                    // vector stores as wide as the row's alignment allows (a row 8 bytes
                    // off a 16-byte boundary -- X even, X % 4 != 0 -- still takes 8-byte
                    // stores at x-spacings 4 and 8)
                    constexpr int DXS = DX > 0 ? DX : 1;
                    constexpr int VW = BF16 ? 1 : tile_vec<DXS>();
                    if (VW == 4 && (shift & 15) == 0) emit_tile<DXS, 4, BF16, C, PK>(sv, p0, p1, p2, p3);
                    else if (VW >= 2 && (shift & 7) == 0) emit_tile<DXS, VW >= 2 ? 2 : 1, BF16, C, PK>(sv, p0, p1, p2, p3);
                    else emit_tile<DXS, 1, BF16, C, PK>(sv, p0, p1, p2, p3);
                } else {
                    for (int r = 0; r < rn; ++r)
                        emit_voxel<BF16, C, PK>(sv + C * ES * r, wxb + 4 * r, p0, p1, p2, p3);
                }
            }
            fence_proxy_async_smem();  // this lane's staging writes before the bulk copy reads them
            __syncwarp();
            BSI_GUARD((g - static_cast<unsigned char*>(d.field)) / ES + (long long)C * u.nvox <=
                              (long long)C * d.X * d.Y * d.Z &&
                          g >= static_cast<unsigned char*>(d.field) && shift + nbytes <= buf_bytes,
                      kErrFieldWrite, err) {
                store_row<ES>(sb, g, shift, nbytes, lane);
            }
            __syncwarp();  // lane 0's ring wait in store_row precedes every lane's next staging write
        }
    }
}

// One forward unit on the tensor-store path (see fwd_tma_rows): the rows of the
// unit's tile-row are staged rb at a time into a block of `stage`'s ring (row
// pitch = the strip's bytes, every row on a 16-byte boundary), and each block
// leaves as one tensor store at (strip start, first row, plane); rows and
// columns past the volume's end are clipped by the copy.  Halo lanes (lane >=
// gcells) stage into the warp's spare slot after the ring.  C = 3 channels
// (the displacement field) or 1 (scalar interpolation).
template <int DX, bool BF16, int C = 3>
__device__ __forceinline__ void forward_unit_tma(const InstDesc& d, const void* tmap, long long ul,
                                                 unsigned char* stage, int blk_bytes, int rb, int lane, int& ring,
                                                 unsigned* err) {
    static_assert(C == 1 || C == 3, "one (scalar) or three (displacement) channels");
    constexpr int ES = BF16 ? 2 : 4;
    constexpr bool PK = fwd_packed<DX, BF16>();
    constexpr int VW = BF16 ? 1 : tile_vec<DX>();
    const FwdUnit u = fwd_unit(d, ul);
    const int col = u.cell0 + lane;
    float ph[4][4][C];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float a = 0.f, b = 0.f, c = 0.f;
            if (col < d.nx) {
                // C channels per control point: [nz][ny][nx][C]
                const long long e = (((long long)(u.kz + n) * d.ny + (u.jy + m)) * d.nx + col) * C;
                BSI_GUARD(e >= 0 && e + C <= (long long)C * d.nx * d.ny * d.nz, kErrPhiRead, err) {
                    const float* p = d.phi + e;
                    a = __ldg(p);
                    if (C == 3) {
                        b = __ldg(p + 1);
                        c = __ldg(p + 2);
                    }
                }
            }
            ph[n][m][0] = a;
            ph[n][m][C > 1 ? 1 : 0] = C > 1 ? b : a;
            ph[n][m][C > 2 ? 2 : 0] = C > 2 ? c : a;
        }

    const int z0 = u.kz * d.dz, zn = imin(d.dz, d.Z - z0);
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const int wzb = weight_base(d.dz), wyb = weight_base(d.dy);
    const int rowb = d.gcells * DX * C * ES;           // row pitch of a block: the strip's bytes
    const int c0 = (u.x0 * C * ES) >> 3;               // strip start in 8-byte elements (even: 16-byte aligned)
    // this lane's tile in row 0 of a block, or the spare slot for halo lanes
    const uint32_t lane_off = lane < d.gcells ? (uint32_t)(lane * DX * C * ES) : (uint32_t)(kStoreStages * blk_bytes);
    BSI_GUARD(rowb * rb <= blk_bytes && (u.x0 * C * ES) % 16 == 0, kErrStage, err) {}

    for (int rz = 0; rz < zn; ++rz) {
        const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
        const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
        float pz[4][C];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            combine4<C, PK>(pz[m], a0, a1, a2, a3, ph[0][m], ph[1][m], ph[2][m], ph[3][m]);

        for (int yb = 0; yb < yn; yb += rb) {
            unsigned char* blk = stage + ring * blk_bytes;
            ring = ring == kStoreStages - 1 ? 0 : ring + 1;
            // (the block is free: the store of the block kStoreStages - 1 earlier has read it)
            const uint32_t sv0 = smem_u32(lane < d.gcells ? blk : stage) + lane_off;
            const int rows = imin(rb, yn - yb);
            for (int r = 0; r < rows; ++r) {
                const int ry = yb + r;
                const float b0 = c_lut.w[wyb + 4 * ry], b1 = c_lut.w[wyb + 4 * ry + 1];
                const float b2 = c_lut.w[wyb + 4 * ry + 2], b3 = c_lut.w[wyb + 4 * ry + 3];
                float p0[C], p1[C], p2[C], p3[C];
                combine4<C, PK>(p0, b0, b1, b2, b3, pz[0], pz[1], pz[2], pz[3]);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    p1[c] = __shfl_down_sync(kFull, p0[c], 1);
                    p2[c] = __shfl_down_sync(kFull, p0[c], 2);
                    p3[c] = __shfl_down_sync(kFull, p0[c], 3);
                }
                // halo lanes write the spare slot again for every row (never copied out)
                const uint32_t sv = sv0 + (lane < d.gcells ? (uint32_t)(r * rowb) : 0u);
                emit_tile<DX, VW, BF16, C, PK, true>(sv, p0, p1, p2, p3);
            }
            fence_proxy_async_smem();  // this lane's staging writes before the tensor store reads them
            __syncwarp();
            if (lane == 0) {
                tensor_store_3d(tmap, c0, y0 + yb, z0 + rz, blk);
                bulk_commit();
                bulk_wait_read<kStoreStages - 1>();
            }
            __syncwarp();  // lane 0's ring wait precedes every lane's next staging write
        }
    }
}

// ------------------------------------------------------------------ adjoint

// Writes one completed grid plane of a unit's partial sums, NR = jrows + 3 grid
// rows (lanes 3..31 hold the 29 complete columns).
template <int NR>
__device__ __forceinline__ void flush_plane(const InstDesc& d, long long ul, int pz, const AdjUnit& u,
                                            int lane, const float (&h)[NR][3], float* part,
                                            long long ws_floats, unsigned* err) {
    const int j = lane - kHalo;
    if (j >= 0 && u.col0 + j < d.nx) {
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            const long long e = part_elem(d, ul, pz, m, j);
            BSI_GUARD(e >= 0 && e + 3 <= ws_floats, kErrPartWrite, err) {
                part[e] = h[m][0];
                part[e + 1] = h[m][1];
                part[e + 2] = h[m][2];
            }
        }
    }
}

// Bulk-load plan of one gradient row segment [g, g + nbytes): the copy covers
// [s0, s1), the 16-byte-aligned superset of the segment clipped to the
// 16-byte-aligned interior [A0, A1) of the gradient array, and lands in the
// ring buffer at offset s0 - floor16(g); element e of the row then sits at
// offset (g - floor16(g)) + 4e.  Bytes of the segment outside [s0, s1) exist
// only at the two ends of the array and are loaded by lanes.
struct RowLoad {
    uintptr_t g, lo, s0, s1;
};

__device__ __forceinline__ RowLoad row_load(const unsigned char* g, int nbytes, uintptr_t A0, uintptr_t A1) {
    RowLoad r;
    r.g = reinterpret_cast<uintptr_t>(g);
    r.lo = floor16(r.g);
    r.s0 = r.lo > A0 ? r.lo : A0;
    const uintptr_t hi = ceil16(r.g + (uintptr_t)nbytes);
    r.s1 = hi < A1 ? hi : A1;
    return r;
}

// q += w (g0, g1, g2): channels 0 and 1 in one packed FP32x2 FMA (bitwise the
// two scalar FMAs), channel 2 in a scalar one.
__device__ __forceinline__ void fma3(float (&q)[3], float w, float g0, float g1, float g2) {
    const float2 a = __ffma2_rn(make_float2(w, w), make_float2(g0, g1), make_float2(q[0], q[1]));
    q[0] = a.x;
    q[1] = a.y;
    q[2] = fmaf(w, g2, q[2]);
}

// q += w (g0, g1, g2) with three scalar FMAs.
__device__ __forceinline__ void fma3_scalar(float (&q)[3], float w, float g0, float g1, float g2) {
    q[0] = fmaf(w, g0, q[0]);
    q[1] = fmaf(w, g1, q[1]);
    q[2] = fmaf(w, g2, q[2]);
}

template <bool PK>
__device__ __forceinline__ void fma3_sel(float (&q)[3], float w, float g0, float g1, float g2) {
    if constexpr (PK) fma3(q, w, g0, g1, g2);
    else fma3_scalar(q, w, g0, g1, g2);
}

// x-transpose of one voxel: q_l += B_l(r/dx) g, per channel; the voxel's three
// channels sit at shared address sv.
template <bool PK = true>
__device__ __forceinline__ void gather_voxel(float (&q4)[4][3], uint32_t sv, int wo) {
    const float g0 = lds_f32(sv), g1 = lds_f32(sv + 4), g2 = lds_f32(sv + 8);
#pragma unroll
    for (int l = 0; l < 4; ++l) fma3_sel<PK>(q4[l], c_lut.w[wo + l], g0, g1, g2);
}

// x-transpose of a whole tile of DX voxels read from shared address sv with
// VW-float loads (sv aligned to 4 VW bytes; see tile_vec).
template <int DX, int VW, bool PK = true>
__device__ __forceinline__ void gather_tile(float (&q4)[4][3], uint32_t sv) {
    if (VW == 1) {
#pragma unroll
        for (int r = 0; r < DX; ++r) gather_voxel<PK>(q4, sv + 12u * r, weight_base(DX) + 4 * r);
    } else {
        float g[3 * DX];
#pragma unroll
        for (int i = 0; i < 3 * DX / VW; ++i) {
            if (VW == 4) lds_v4_f32(sv + 16 * i, g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
            else lds_v2_f32(sv + 8 * i, g[2 * i], g[2 * i + 1]);
        }
#pragma unroll
        for (int r = 0; r < DX; ++r)
#pragma unroll
            for (int l = 0; l < 4; ++l)
                fma3_sel<PK>(q4[l], c_lut.w[weight_base(DX) + 4 * r + l], g[3 * r], g[3 * r + 1], g[3 * r + 2]);
    }
}

// Column sum and y-stage of one row: the column of lane l collects q4[k] of the
// tile k lanes below, h = ((q4[0] + q4[1]') + q4[2]'') + q4[3]''' per channel,
// and hy[OFF + m] += b_m h (OFF: the row's tile-row within the unit); channels
// 0 and 1 packed (bitwise the scalar form).
template <int OFF = 0, int NR = 4>
__device__ __forceinline__ void column_sum_y(const float (&q4)[4][3], float (&hy)[NR][3], float b0, float b1,
                                             float b2, float b3) {
    static_assert(OFF + 4 <= NR, "four grid rows from OFF");
    float s1[3], s2[3], s3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s1[c] = __shfl_up_sync(kFull, q4[1][c], 1);
        s2[c] = __shfl_up_sync(kFull, q4[2][c], 2);
        s3[c] = __shfl_up_sync(kFull, q4[3][c], 3);
    }
    float2 h = __fadd2_rn(make_float2(q4[0][0], q4[0][1]), make_float2(s1[0], s1[1]));
    h = __fadd2_rn(h, make_float2(s2[0], s2[1]));
    h = __fadd2_rn(h, make_float2(s3[0], s3[1]));
    const float h2 = q4[0][2] + s1[2] + s2[2] + s3[2];
    fma3(hy[OFF], b0, h.x, h.y, h2);
    fma3(hy[OFF + 1], b1, h.x, h.y, h2);
    fma3(hy[OFF + 2], b2, h.x, h.y, h2);
    fma3(hy[OFF + 3], b3, h.x, h.y, h2);
}

// z-stage of one voxel plane: hz[n][m] += a_n hy[m] over the unit's NR grid rows.
template <int NR>
__device__ __forceinline__ void accumulate_z(float (&hz)[4][NR][3], const float (&hy)[NR][3], float a0, float a1,
                                             float a2, float a3) {
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        fma3(hz[0][m], a0, hy[m][0], hy[m][1], hy[m][2]);
        fma3(hz[1][m], a1, hy[m][0], hy[m][1], hy[m][2]);
        fma3(hz[2][m], a2, hy[m][0], hy[m][1], hy[m][2]);
        fma3(hz[3][m], a3, hy[m][0], hy[m][1], hy[m][2]);
    }
}

template <int DX>
__device__ __forceinline__ bool adjoint_unit(const InstDesc& d, long long ul, uint64_t* bars,
                                             unsigned char* bufs, int buf_bytes, int lane, unsigned& q,
                                             float* part, long long ws_floats, unsigned* err) {
    const int dx = DX > 0 ? DX : d.dx;
    const AdjUnit u = adj_unit(d, ul);
    const int cell = u.col0 - kHalo + lane;
    const int nv = (cell >= 0 && cell < d.ncx) ? imin(dx, d.X - cell * dx) : 0;
    // A specialised spacing reads all DX voxels of every lane, unpredicated.  In
    // a ragged unit (a cut or empty tile: the first and last x-groups) each
    // staged row gets zfloats zeros right after its nvox voxels; a cut tile
    // reads its missing voxels there and an empty tile reads all of its voxels
    // there, so both add exact zeros.  The zeros end by voxel 32 DX of the
    // strip, inside the ring buffer.
    const bool ragged = DX > 0 && !__all_sync(kFull, nv == dx);
    const int zfloats = 3 * imin(dx, kLanes * dx - u.nvox);
    // strip-local first voxel of this lane's tile (empty tiles: the zeros)
    const int xl = (DX > 0 && nv == 0) ? u.nvox : cell * dx - u.xs;
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const int zb = u.kz0 * d.dz;
    const int rows = (imin(u.kz1 * d.dz, d.Z) - zb) * yn;
    const int wxb = weight_base(dx), wyb = weight_base(d.dy), wzb = weight_base(d.dz);
    const int nbytes = u.nvox * 12;
    const long long row_pitch = 12LL * d.X;              // bytes from row y to row y + 1
    const long long plane_pitch = row_pitch * d.Y;       // bytes from plane z to plane z + 1
    const uintptr_t gbase = reinterpret_cast<uintptr_t>(d.grad);
    const uintptr_t A0 = ceil16(gbase);
    const uintptr_t A1 = floor16(gbase + (uintptr_t)(12LL * d.X * d.Y * d.Z));
    const uintptr_t g_first = gbase + 4 * field_elem(d, zb, y0, u.xs);   // row 0 of the unit
    // only a unit holding the first or last row of the array has bytes outside the bulk copies
    const bool unit_edge = g_first < A0 ||
        gbase + 4 * field_elem(d, imin(u.kz1 * d.dz, d.Z) - 1, y0 + yn - 1, u.xs) + (uintptr_t)nbytes > A1;
    const unsigned q0 = q;

    // Producer (lane 0): puts the unit's rows in flight in order, row k into ring
    // buffer (q0 + k) % kLoadStages; ig / iy / ik track the next row to issue.
    uintptr_t ig = g_first;
    int iy = 0, ik = 0;
    auto issue_next = [&]() {
        const unsigned st = (q0 + (unsigned)ik) % kLoadStages;
        const RowLoad L = row_load(reinterpret_cast<const unsigned char*>(ig), nbytes, A0, A1);
        if (L.s1 > L.s0) {
            mbar_arrive_expect_tx(&bars[st], (uint32_t)(L.s1 - L.s0));
            bulk_load(bufs + st * buf_bytes + (L.s0 - L.lo), reinterpret_cast<const void*>(L.s0),
                      (uint32_t)(L.s1 - L.s0), &bars[st]);
        } else {
            mbar_arrive(&bars[st]);
        }
        ++ik;
        ig += row_pitch;
        if (++iy == yn) {
            iy = 0;
            ig += plane_pitch - yn * row_pitch;
        }
    };
    if (lane == 0)
        for (int k = 0; k < rows && k < kLoadStages; ++k) issue_next();
    uintptr_t gz = g_first;   // consumer: first row of the current voxel plane

    float hz[4][4][3];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[n][m][c] = 0.f;

    int k = 0;
    for (int kz = u.kz0; kz < u.kz1; ++kz) {
        const int z0 = kz * d.dz, zn = imin(d.dz, d.Z - z0);
        for (int rz = 0; rz < zn; ++rz, gz += plane_pitch) {
            float hy[4][3];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hy[m][c] = 0.f;

            uintptr_t g = gz;
            for (int ry = 0; ry < yn; ++ry, ++k, g += row_pitch) {
                const unsigned qq = q0 + (unsigned)k;
                const unsigned st = qq % kLoadStages;
                if (!mbar_wait_bounded(&bars[st], (qq / kLoadStages) & 1u)) {
                    // a bulk copy never completed: record it, give the copies still
                    // in flight a bounded chance to land, and stop this warp
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    for (int p = k + 1; p < rows && p < k + kLoadStages; ++p) {
                        const unsigned qp = q0 + (unsigned)p;
                        (void)mbar_wait_bounded(&bars[qp % kLoadStages], (qp / kLoadStages) & 1u);
                    }
                    q = q0 + (unsigned)rows;
                    return false;
                }
                unsigned char* sb = bufs + st * buf_bytes + (g & 15);
                BSI_GUARD((int)(g & 15) + nbytes <= buf_bytes && g >= gbase &&
                              (long long)(g - gbase) / 4 + 3LL * u.nvox <= 3LL * d.X * d.Y * d.Z,
                          kErrGradRead, err) {
                    if (unit_edge && (g < A0 || g + (uintptr_t)nbytes > A1)) {
                        // first or last row of the array: elements outside the bulk copy
                        const RowLoad L = row_load(reinterpret_cast<const unsigned char*>(g), nbytes, A0, A1);
                        for (int i = lane; i < u.nvox * 3; i += kLanes) {
                            const uintptr_t a = g + 4u * (uintptr_t)i;
                            if (a < L.s0 || a >= L.s1)
                                reinterpret_cast<float*>(sb)[i] = *reinterpret_cast<const float*>(a);
                        }
                    }
                }
                BSI_GUARD((int)(g & 15) + 12 * u.nvox + 4 * zfloats <= buf_bytes, kErrStage, err) {
                    if (ragged && lane < zfloats) sts_f32(smem_u32(sb) + 12u * (uint32_t)u.nvox + 4u * lane, 0.f);
                }
                __syncwarp();
                // shared address of this lane's first voxel
                const uint32_t sv = smem_u32(sb) + 12u * (uint32_t)xl;
                float q4[4][3];
#pragma unroll
                for (int l = 0; l < 4; ++l)
#pragma unroll
                    for (int c = 0; c < 3; ++c) q4[l][c] = 0.f;
                if (DX > 0) {  // one path for all lanes: full, cut and empty tiles
                    constexpr int DXS = DX > 0 ? DX : 1;
                    // 16-byte loads for DX = 4, 8 (8-byte loads for DX = 2, 6 measured slower
                    // than scalar ones)
                    constexpr int VW = DXS % 4 == 0 ? 4 : 1;
                    // vector loads when every lane's start is aligned (warp-uniform): the
                    // row start, and in a ragged unit the zeros after nvox voxels
                    const uint32_t amask = 4 * VW - 1;
                    if (VW > 1 && ((uint32_t)g & amask) == 0 && (!ragged || ((12u * u.nvox) & amask) == 0))
                        gather_tile<DXS, VW>(q4, sv);
                    else
                        gather_tile<DXS, 1>(q4, sv);
                } else {
                    for (int r = 0; r < nv; ++r) gather_voxel(q4, sv + 12u * r, wxb + 4 * r);
                }
                // this ring buffer may be refilled once every lane has read it
                fence_proxy_async_smem();
                __syncwarp();
                // refill in pairs: after every second row the two freed ring buffers
                // get the next two rows, one lane-0 block for both copies
                if (lane == 0 && (k & 1) && ik < rows) {
                    issue_next();
                    if (ik < rows) issue_next();
                }

                // column sum: the column of lane l collects q4[k] of the tile k lanes below
                const float b0 = c_lut.w[wyb + 4 * ry], b1 = c_lut.w[wyb + 4 * ry + 1];
                const float b2 = c_lut.w[wyb + 4 * ry + 2], b3 = c_lut.w[wyb + 4 * ry + 3];
                column_sum_y(q4, hy, b0, b1, b2, b3);
            }
            const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
            const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
            accumulate_z(hz, hy, a0, a1, a2, a3);
        }
        // grid plane kz is complete for this unit; roll the window by one plane
        flush_plane(d, ul, kz - u.kz0, u, lane, hz[0], part, ws_floats, err);
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hz[n][m][c] = hz[n + 1][m][c];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[3][m][c] = 0.f;
    }
    const int nk = u.kz1 - u.kz0;
#pragma unroll
    for (int n = 0; n < 3; ++n) flush_plane(d, ul, nk + n, u, lane, hz[n], part, ws_floats, err);
    q = q0 + (unsigned)rows;
    return true;
}

// One adjoint unit on the tensor-copy path (see tma_boxes), JR tile-rows (1 or
// 2; with 2 a control point's partial sums overlap over 2.5 units in y instead
// of 4, so fewer partial sums are written and reduced): block k of the
// unit (rows [i rb, i rb + rb) of voxel plane p, k = p * nblk + i) arrives as
// one or two boxes in ring stage (q0 + k) % stages, issued `stages` blocks
// ahead by lane 0; a warp waits once per block.  Halo, cut and empty tiles read
// the zeros the copy fills in outside the array, so every lane runs the same
// unpredicated code.  Rows are summed in the same order as adjoint_unit.
// The tensor-copy adjoint's x-transpose stays scalar (its y and z stages are
// packed): packed, that kernel alone ran 2% faster on a 512 x 512 x 300 volume
// at spacing 5, but a forward + adjoint step 0.8% slower (0.3254 -> 0.3280 ms,
// three interleaved runs), where the adjoint is bound by its reads.
constexpr bool kTmaGatherPacked = false;

template <int DX, int JR>
__device__ __forceinline__ bool adjoint_unit_tma(const InstDesc& d, const void* tmap, long long ul,
                                                 uint64_t* bars, unsigned char* ring, int stage_bytes, int stages,
                                                 int lane, unsigned& q, float* part, long long ws_floats,
                                                 unsigned* err) {
    const AdjUnit u = adj_unit(d, ul);
    constexpr int NB = DX <= 5 ? 1 : 2;                     // tma_boxes(DX)
    constexpr int W = NB == 1 ? 48 * DX + 2 : 24 * DX + 2;  // tma_box_width(DX), 8-byte elements
    constexpr int row_bytes = 8 * W;
    const int rb = d.tma_rows;
    const int box_pad = (row_bytes * rb + 127) & ~127;      // tma_box_bytes(DX, rb)
    const int f0 = tma_first_float(u, DX);
    const int gx0 = tma_group_of(f0);
    const int shift = f0 - 4 * gx0;                         // 0..3 floats
    constexpr int NR = JR + kHalo;                          // grid rows the unit's sums reach
    const int y0 = u.jy * d.dy, yn = imin(JR * d.dy, d.Y - y0);
    const int nblk = (yn + rb - 1) / rb;                    // blocks per voxel plane of the unit's tile-rows
    const int zb = u.kz0 * d.dz;
    const int planes = imin(u.kz1 * d.dz, d.Z) - zb;
    const int blocks = planes * nblk;
    const uint32_t block_bytes = (uint32_t)(NB * row_bytes * rb);
    const int wyb = weight_base(d.dy), wzb = weight_base(d.dz);
    const unsigned q0 = q;
    BSI_GUARD(rb >= 1 && rb <= kTmaMaxRows && NB * box_pad <= stage_bytes && shift + 3 * DX * (kLanes / NB) <= 2 * W,
              kErrStage, err) {}

    // producer (lane 0): next block to put in flight, as (plane, block in plane)
    int ik = 0, ip = 0, ii = 0;
    auto issue = [&]() {
        const unsigned st = (q0 + (unsigned)ik) % (unsigned)stages;
        mbar_arrive_expect_tx(&bars[st], block_bytes);
#pragma unroll
        for (int bx = 0; bx < NB; ++bx)   // box bx starts 48 DX floats (24 DX elements) after box bx - 1
            tensor_load_3d(ring + st * stage_bytes + bx * box_pad, tmap, 2 * gx0 + bx * 24 * DX, y0 + ii * rb,
                           zb + ip, &bars[st]);
        ++ik;
        if (++ii == nblk) {
            ii = 0;
            ++ip;
        }
    };
    if (lane == 0)
        while (ik < blocks && ik < stages) issue();
    const int bl = NB == 1 ? 0 : lane >> 4;                // this lane's box
    const uint32_t lane_off = (uint32_t)(bl * box_pad) + 4u * (uint32_t)shift + 12u * DX * (uint32_t)(lane - 16 * bl);

    float hz[4][NR][3];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < NR; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[n][m][c] = 0.f;

    int k = 0;
    for (int kz = u.kz0; kz < u.kz1; ++kz) {
        const int z0 = kz * d.dz, zn = imin(d.dz, d.Z - z0);
        for (int rz = 0; rz < zn; ++rz) {
            float hy[NR][3];
#pragma unroll
            for (int m = 0; m < NR; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hy[m][c] = 0.f;
            for (int i = 0; i < nblk; ++i, ++k) {
                const unsigned qq = q0 + (unsigned)k;
                const unsigned st = qq % (unsigned)stages;
                if (!mbar_wait_bounded(&bars[st], (qq / (unsigned)stages) & 1u)) {
                    // a block never completed: record it, give the blocks still in
                    // flight a bounded chance to land, and stop this warp
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    for (int kk = k + 1; kk < blocks && kk < k + stages; ++kk) {
                        const unsigned qp = q0 + (unsigned)kk;
                        (void)mbar_wait_bounded(&bars[qp % (unsigned)stages], (qp / (unsigned)stages) & 1u);
                    }
                    q = q0 + (unsigned)blocks;
                    return false;
                }
                // shared address of this lane's first voxel in row 0 of the block
                const uint32_t sv = smem_u32(ring + st * stage_bytes) + lane_off;
                const int ry0 = i * rb, rows = imin(rb, yn - ry0);
                for (int r = 0; r < rows; ++r) {
                    const int ry = ry0 + r;
                    float q4[4][3];
#pragma unroll
                    for (int l = 0; l < 4; ++l)
#pragma unroll
                        for (int c = 0; c < 3; ++c) q4[l][c] = 0.f;
                    // 16-byte loads for DX = 4, 8: shift is then 0, box rows are 16-byte multiples
                    gather_tile<DX, DX % 4 == 0 ? 4 : 1, kTmaGatherPacked>(q4, sv + (uint32_t)(r * row_bytes));
                    // the row's tile-row within the unit (0 or 1) and its offset in that tile-row
                    const int t = (JR > 1 && ry >= d.dy) ? 1 : 0;
                    const int rr = ry - t * d.dy;
                    const float b0 = c_lut.w[wyb + 4 * rr], b1 = c_lut.w[wyb + 4 * rr + 1];
                    const float b2 = c_lut.w[wyb + 4 * rr + 2], b3 = c_lut.w[wyb + 4 * rr + 3];
                    if constexpr (JR > 1) {
                        if (t) column_sum_y<1>(q4, hy, b0, b1, b2, b3);
                        else column_sum_y<0>(q4, hy, b0, b1, b2, b3);
                    } else {
                        column_sum_y<0>(q4, hy, b0, b1, b2, b3);
                    }
                }
                // the stage may be refilled once every lane has read it
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && ik < blocks) issue();
            }
            const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
            const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
            accumulate_z(hz, hy, a0, a1, a2, a3);
        }
        flush_plane(d, ul, kz - u.kz0, u, lane, hz[0], part, ws_floats, err);
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < NR; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hz[n][m][c] = hz[n + 1][m][c];
#pragma unroll
        for (int m = 0; m < NR; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[3][m][c] = 0.f;
    }
    const int nk = u.kz1 - u.kz0;
#pragma unroll
    for (int n = 0; n < 3; ++n) flush_plane(d, ul, nk + n, u, lane, hz[n], part, ws_floats, err);
    q = q0 + (unsigned)blocks;
    return true;
}

}  // namespace bsi
