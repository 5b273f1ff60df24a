// bsi_abi.cu -- the C ABI declared in include/bsi.h: host-side validation,
// launch planning and the host-only range self-check.
#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "bsi.h"
#include "bsi_geometry.h"
#include "bsi_launch.h"

namespace bsi {

// ----------------------------------------------------------- kernel facts

cudaError_t kernel_facts(const void* kernel, int threads, int smem, KernelFacts* out) {
    static std::mutex mu;
    struct Key {
        const void* k;
        int dev, threads, smem;
        bool operator==(const Key& o) const {
            return k == o.k && dev == o.dev && threads == o.threads && smem == o.smem;
        }
    };
    struct KeyHash {
        size_t operator()(const Key& a) const {
            return std::hash<const void*>()(a.k) ^ ((size_t)a.dev << 40) ^ ((size_t)a.threads << 20) ^
                   (size_t)a.smem;
        }
    };
    static std::unordered_map<Key, KernelFacts, KeyHash> cache;
    // The dynamic shared-memory limit is an attribute of the kernel, not of a
    // launch: it is only ever raised, to the largest size requested so far.
    static std::unordered_map<Key, int, KeyHash> smem_limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const Key key{kernel, dev, threads, smem};
    const Key kkey{kernel, dev, 0, 0};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    KernelFacts f;
    e = cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    auto lim = smem_limit.find(kkey);
    const int have = lim == smem_limit.end() ? 48 * 1024 : lim->second;
    if (smem > have) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        smem_limit[kkey] = smem;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f.ctas_per_sm, kernel, threads, (size_t)smem);
    if (e != cudaSuccess) return e;
    if (f.ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
    cache.emplace(key, f);
    *out = f;
    return cudaSuccess;
}

// ----------------------------------------------------------- planning

// Tile-planes per adjoint unit: kMinZChunk..kMaxZChunk, chosen per volume by
// choose_zchunk unless the tile-config table fixes it.  Must be >= 3: the
// reduce kernel then finds every grid plane in at most two consecutive chunks.
constexpr int kMinZChunk = 3;
constexpr int kMaxZChunk = 16;
constexpr int kDefaultZChunk = 4;   // where no model applies (empty volumes, workspace queries)
static_assert(kMinZChunk >= 3, "adjoint reduce assumes chunks of at least 3 tile-planes");

static thread_local char t_cuda_msg[256] = "";

static bsi_status cuda_fail(cudaError_t e) {
    std::snprintf(t_cuda_msg, sizeof t_cuda_msg, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return BSI_ERR_CUDA;
}

static bsi_status check_geom(const bsi_geom* g) {
    if (!g) return BSI_ERR_NULL;
    if (g->X < 0 || g->Y < 0 || g->Z < 0 || g->X > BSI_MAX_DIM || g->Y > BSI_MAX_DIM || g->Z > BSI_MAX_DIM)
        return BSI_ERR_DIMS;
    if (g->dx < 1 || g->dy < 1 || g->dz < 1 || g->dx > BSI_MAX_SPACING || g->dy > BSI_MAX_SPACING ||
        g->dz > BSI_MAX_SPACING)
        return BSI_ERR_SPACING;
    if (g->nx != cdiv(g->X, g->dx) + 3 || g->ny != cdiv(g->Y, g->dy) + 3 || g->nz != cdiv(g->Z, g->dz) + 3)
        return BSI_ERR_GRID_MISMATCH;
    return BSI_OK;
}

static bool empty_volume(const bsi_geom& g) { return g.X == 0 || g.Y == 0 || g.Z == 0; }

// ----------------------------------------------------------- tile-config table

static std::mutex g_cfg_mu;
static std::vector<bsi_tile_config> g_cfg;

static bool config_valid(const bsi_tile_config& c) {
    auto sp = [](int32_t v) { return v == 0 || (v >= 1 && v <= BSI_MAX_SPACING); };
    return sp(c.dx) && sp(c.dy) && sp(c.dz) && (c.adj_zchunk == 0 || (c.adj_zchunk >= 3 && c.adj_zchunk <= 16)) &&
           (c.fwd_strip_tiles == 0 || (c.fwd_strip_tiles >= 4 && c.fwd_strip_tiles <= kGroupCells)) &&
           (c.adj_warps >= 0 && c.adj_warps <= kAdjWarpsMax) &&
           (c.fwd_warps >= 0 && c.fwd_warps <= kMaxWarpsPerCta);
}

// The table entry for spacing (dx, dy, dz) with zero fields left as they are
// (the caller applies the defaults), or an all-zero config if none matches.
static bsi_tile_config lookup_config(int32_t dx, int32_t dy, int32_t dz) {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    for (const bsi_tile_config& c : g_cfg)
        if ((c.dx == 0 || c.dx == dx) && (c.dy == 0 || c.dy == dy) && (c.dz == 0 || c.dz == dz)) return c;
    bsi_tile_config z;
    std::memset(&z, 0, sizeof z);
    return z;
}

static void fill_desc(InstDesc& d, const bsi_geom& g, bool adjoint, bool bf16 = false) {
    const bsi_tile_config cfg = lookup_config(g.dx, g.dy, g.dz);
    const int zchunk = cfg.adj_zchunk > 0 ? cfg.adj_zchunk : kDefaultZChunk;
    std::memset(&d, 0, sizeof d);
    d.warps_req = adjoint ? cfg.adj_warps : cfg.fwd_warps;
    d.X = (int)g.X;
    d.Y = (int)g.Y;
    d.Z = (int)g.Z;
    d.dx = g.dx;
    d.dy = g.dy;
    d.dz = g.dz;
    d.nx = (int)g.nx;
    d.ny = (int)g.ny;
    d.nz = (int)g.nz;
    const bool empty = empty_volume(g);
    if (!empty) {
        d.ncx = (int)cdiv(g.X, g.dx);
        d.ncy = (int)cdiv(g.Y, g.dy);
        d.ncz = (int)cdiv(g.Z, g.dz);
    }
    d.jrows = 1;
    d.ncyu = d.ncy;
    if (!adjoint) {
        d.gcells = cfg.fwd_strip_tiles > 0 ? cfg.fwd_strip_tiles : fwd_strip_tiles(d.X, d.dx, bf16);
        d.nxg = empty ? 0 : (int)cdiv(d.ncx, d.gcells);
        d.units = (long long)d.ncz * d.ncy * d.nxg;
    } else {
        d.zchunk = zchunk;
        d.tma_rows = tma_block_rows(d.dx, d.dy);
        d.nxg = empty ? 0 : (int)cdiv(d.nx, kGroupCells);
        d.nzc = empty ? 0 : (int)cdiv(d.ncz, zchunk);
        d.units = (long long)d.nzc * d.ncyu * d.nxg;
    }
}

static void set_zchunk(InstDesc& d, int zc) {
    d.zchunk = zc;
    d.nzc = d.ncz > 0 ? (int)cdiv(d.ncz, zc) : 0;
    d.units = (long long)d.nzc * d.ncyu * d.nxg;
}

// Tile-rows per adjoint unit on the tensor-copy path where taken (the row path
// takes 1): two tile-rows cut the partial sums' overlap in y from 4 units to
// 2.5, so fewer are written and reduced.  Taken for single-volume calls at
// y-spacings 4..6, where it measured faster (512 x 512 x 300 at spacing 5: the
// forward + adjoint step 0.3192 -> 0.3140 ms; 512^3 at 4: 0.346 -> 0.326 ms,
// at (6,5,4): 0.302 -> 0.274 ms), and not at y-spacing 3 (+1.5%: the 11-warp
// register budget of two-row units) or 8 (+8.6%), nor in batches (a launch
// more; +6% for the 64-volume batch).
constexpr int kTmaJrows = 2;
constexpr int kTmaJrowsMinDy = 4, kTmaJrowsMaxDy = 6;
static bool two_row_units(const InstDesc& d, int n) {
    return kTmaJrows > 1 && n == 1 && d.dy >= kTmaJrowsMinDy && d.dy <= kTmaJrowsMaxDy;
}

static void set_jrows(InstDesc& d, int jr) {
    d.jrows = jr;
    d.ncyu = d.ncy > 0 ? (int)cdiv(d.ncy, jr) : 0;
    d.units = (long long)d.nzc * d.ncyu * d.nxg;
}

static long long adj_floats(const InstDesc& d) {
    const long long f = d.units * adj_unit_floats(d);
    return (f + 3) & ~3LL;  // keep every instance's partials 16-byte aligned
}

// Workspace floats an adjoint instance may need: the most (least, with
// `least`) over every plan the launch may pick -- tile-rows per unit 1, or also
// kTmaJrows where the volume could take the tensor-copy path, times the table's
// zchunk if it fixes one, else every zchunk choose_zchunk may pick.
static long long adj_floats_bound(const bsi_geom& g, bool least = false) {
    InstDesc d;
    fill_desc(d, g, true);
    const bool fixed = lookup_config(g.dx, g.dy, g.dz).adj_zchunk > 0;
    const int jrs[2] = {1, kTmaJrows};
    const int njr = (two_row_units(d, 1) && d.units > 0 && d.dx <= kMaxSpecializedDx && d.X % 4 == 0) ? 2 : 1;
    long long m = -1;
    for (int k = 0; k < njr; ++k) {
        set_jrows(d, jrs[k]);
        for (int zc = kMinZChunk; zc <= kMaxZChunk; ++zc) {
            if (!fixed) set_zchunk(d, zc);
            const long long f = adj_floats(d);
            if (m < 0 || (least ? f < m : f > m)) m = f;
            if (fixed) break;
        }
    }
    return m;
}

// SM count of the current device, cached per device (152, a GB300's, when no
// device can be queried: the host-only self-check).
static int device_sms() {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 152;
    }
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = 152;
    }
    cache.emplace(dev, n);
    return n;
}

// Tile-planes per adjoint unit for one volume by a cost model of the partials
// kernel plus the reduce.  Units run in rounds over the launch's warp slots
// (SMs x warps per SM); a last, partial round costs about as long as
// (0.6 + 0.4 x its fill) of a full one (a lone warp per SM runs faster, not
// proportionally so).  Per zchunk zc:
//   T = rounds / (units / slots) * (gradient + partial bytes) * (1 + 0.3 / zc)
//       + partial bytes (read back by the reduce),
// 0.3 tile-planes being the start-up and flush cost of a unit.  Measured on
// the GPU the model ranks the good and bad choices of 512^3 / 512^2 x 300
// volumes at spacings 3, 5 and 8 correctly to within a few per cent.
// Only plans of at most max_floats partial floats are considered (when >= 0);
// if none fits, the smallest plan.
static int choose_zchunk(const InstDesc& d0, bool tma, long long max_floats = -1) {
    if (d0.ncz <= 0 || d0.units <= 0) return kDefaultZChunk;
    int wps = 3 * kAdjWarpsMax;   // row path: three 4-warp CTAs per SM
    if (tma) {
        const int blk = tma_block_bytes(d0.dx, d0.tma_rows);
        wps = tma_warps_per_cta(blk, tma_default_stages(blk), 0, d0.jrows);
    }
    const double slots = (double)device_sms() * wps;
    const double grad_bytes = 12.0 * d0.X * d0.Y * d0.Z;
    InstDesc d = d0;
    int best = -1, smallest = kDefaultZChunk;
    double best_t = 0;
    long long smallest_f = -1;
    for (int zc = kMinZChunk; zc <= kMaxZChunk; ++zc) {
        set_zchunk(d, zc);
        if (smallest_f < 0 || adj_floats(d) < smallest_f) {
            smallest_f = adj_floats(d);
            smallest = zc;
        }
        if (max_floats >= 0 && adj_floats(d) > max_floats) continue;
        const double n = (double)d.units / slots;
        const double full = (double)(long long)n, f = n - full;
        const double rounds = full + (f > 1e-9 ? 0.6 + 0.4 * f : 0.0);
        const double part_bytes = 4.0 * (double)adj_floats(d);
        const double t = rounds / n * (grad_bytes + part_bytes) * (1.0 + 0.3 / (zc * d.jrows)) + part_bytes;
        if (best < 0 || t < best_t) {
            best = zc;
            best_t = t;
        }
    }
    return best < 0 ? smallest : best;
}

// A launch group: up to kMaxBatch instances that share a kernel variant.
struct Group {
    bool generic = false;
    bool tma = false;    // adjoint tensor-copy path
    int dxmax = 1;
    int tma_stage = 0;   // tensor-copy path: bytes of one ring stage (largest block of its instances)
    int warps_req = 0;   // smallest non-zero warps_per_cta request of its instances
    std::vector<InstDesc> inst;
};

static bool misaligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; }

// Whether an adjoint instance can take the tensor-copy path: rows of 16-byte
// multiples in a 16-byte-aligned array and x-spacing <= 8.
static bool tma_geometry_ok(const InstDesc& d) {
    return d.units > 0 && d.dx <= kMaxSpecializedDx && d.X % 4 == 0 && !misaligned(d.grad, 16);
}

// Splits instances into groups of one kernel variant, in caller order, at most
// kMaxBatch per group: with allow_tma, adjoint instances that can take the
// tensor-copy path (tma_geometry_ok); then x-spacing <= 8 (the
// compile-time-specialised kernel); then larger spacings (the generic one).
// Fills unit/point prefixes and partial offsets.
static std::vector<Group> plan(const std::vector<InstDesc>& all, long long* ws_floats, bool allow_tma = false) {
    std::vector<Group> out;
    long long off = 0;
    // passes: tensor-copy instances with 1, then kTmaJrows tile-rows per unit (one
    // kernel instantiation each), the row path, the generic kernel
    for (int pass = 0; pass < 4; ++pass) {
        const bool tma = pass < 2, generic = pass == 3;
        const int jr = pass == 1 ? kTmaJrows : 1;
        if ((tma && !allow_tma) || (pass == 1 && kTmaJrows == 1)) continue;
        Group cur;
        cur.generic = generic;
        cur.tma = tma;
        for (const InstDesc& d0 : all) {
            const bool t = allow_tma && tma_geometry_ok(d0);
            if (t != tma || (t && d0.jrows != jr) || (!t && (d0.dx > kMaxSpecializedDx) != generic)) continue;
            InstDesc d = d0;
            d.part_off = off;
            off += adj_floats(d);
            cur.inst.push_back(d);
            cur.dxmax = std::max(cur.dxmax, d.dx);
            if (tma) cur.tma_stage = std::max(cur.tma_stage, tma_block_bytes(d.dx, d.tma_rows));
            if (d.warps_req > 0 && (cur.warps_req == 0 || d.warps_req < cur.warps_req)) cur.warps_req = d.warps_req;
            if ((int)cur.inst.size() == kMaxBatch) {
                out.push_back(cur);
                cur.inst.clear();
                cur.dxmax = 1;
                cur.tma_stage = 0;
                cur.warps_req = 0;
            }
        }
        if (!cur.inst.empty()) out.push_back(cur);
    }
    // Heaviest units first within a launch: units are dealt round-robin over the
    // warp slots, so rounds of similar cost keep the warps balanced (unit cost
    // ~ rows x (voxels per lane row + per-row work); for a batch of uneven
    // spacings it varies ~7x; measured +3% on the 64-volume batch).  Instance
    // order never changes any result.
    auto unit_cost = [](const InstDesc& d) {
        const long long planes = d.zchunk > 0 ? (long long)d.zchunk * d.dz : d.dz;
        return planes * d.jrows * d.dy * (d.dx + 4);
    };
    for (Group& g : out)
        std::stable_sort(g.inst.begin(), g.inst.end(),
                         [&](const InstDesc& a, const InstDesc& b) { return unit_cost(a) > unit_cost(b); });
    for (Group& g : out) {
        long long ub = 0, pb = 0;
        for (InstDesc& d : g.inst) {
            d.unit_begin = ub;
            d.point_begin = pb;
            ub += d.units;
            pb += (long long)d.nx * d.ny * d.nz;
        }
    }
    if (ws_floats) *ws_floats = off;
    return out;
}

template <int MAXB>
static void to_batch(const Group& g, Batch<MAXB>& b) {
    std::memset(&b, 0, sizeof b);
    b.n = (int)g.inst.size();
    b.buf_bytes = g.tma ? g.tma_stage : stage_buf_bytes(g.dxmax);
    b.stages = g.tma ? tma_default_stages(g.tma_stage) : 0;
    b.warps_req = g.tma ? 0 : g.warps_req;
    for (int i = 0; i < b.n; ++i) {
        b.inst[i] = g.inst[i];
        b.total_units += g.inst[i].units;
        b.total_points += (long long)g.inst[i].nx * g.inst[i].ny * g.inst[i].nz;
    }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against
// the driver library); null when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The gradient of one instance as a 3-D tensor of 8-byte elements (float
// pairs): (3X/2, Y, Z), with a box of (tma_box_width(dx), tma_rows, 1); zeros
// outside.
static cudaError_t encode_grad_map(const InstDesc& d, CUtensorMap* m) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)d.X * 3 / 2, (cuuint64_t)d.Y, (cuuint64_t)d.Z};
    const cuuint64_t strides[2] = {(cuuint64_t)d.X * 12, (cuuint64_t)d.X * 12 * (cuuint64_t)d.Y};
    const cuuint32_t box[3] = {(cuuint32_t)tma_box_width(d.dx), (cuuint32_t)d.tma_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float*>(d.grad), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The field of one instance as a 3-D tensor of 8-byte elements: (3 X ES / 8,
// Y, Z), with a box of (the strip's bytes / 8, rb, 1) for the forward's
// tensor stores (fwd_tma_rows).
static cudaError_t encode_field_map(const InstDesc& d, bool bf16, int rb, CUtensorMap* m, int c = 3) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t es = bf16 ? 2 : 4;
    const cuuint64_t row = (cuuint64_t)d.X * (cuuint64_t)c * es;
    const cuuint64_t dims[3] = {row / 8, (cuuint64_t)d.Y, (cuuint64_t)d.Z};
    const cuuint64_t strides[2] = {row, row * (cuuint64_t)d.Y};
    const cuuint32_t box[3] = {(cuuint32_t)(fwd_tma_row_bytes(d.gcells, d.dx, bf16, c) / 8), (cuuint32_t)rb, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, d.field, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// BF16 at odd x-spacings >= 5: rows leave by tensor stores when strips of 24
// tiles (g dx a multiple of 8: rows on 16-byte boundaries) take the place of the
// default 29, whose rows end off 16-byte boundaries (512 x 512 x 300 at spacing
// 5: 0.153 -> 0.146 ms; at spacing 3 the idle lanes cost more: 512^3 0.414 ->
// 0.429 ms, not taken).  Re-plans d's strips; true when it did.
static bool bf16_odd_strips(InstDesc& d, bool bf16, bool generic) {
    if (!bf16 || generic || !(d.dx & 1) || d.dx < 5 || d.gcells != kGroupCells || d.units <= 0 ||
        fwd_tma_rows(d.X, d.dx, d.dy, kBf16OddStripTiles, true) <= 0)
        return false;
    d.gcells = kBf16OddStripTiles;
    d.nxg = (int)cdiv(d.ncx, d.gcells);
    d.units = (long long)d.ncz * d.ncy * d.nxg;
    return true;
}

// Rows per block when a single-volume forward of c channels takes the
// tensor-store path, else 0.
static int forward_tma_rows(const InstDesc& d, bool bf16, bool generic, int c = 3) {
    if (generic || d.units <= 0 || (reinterpret_cast<uintptr_t>(d.field) & 15) != 0 || !tensor_map_encoder())
        return 0;
    return fwd_tma_rows(d.X, d.dx, d.dy, d.gcells, bf16, c);
}

enum class Op { Forward, AdjointPartials, AdjointReduce };

template <int MAXB>
static cudaError_t run_partials_tma(const Group& g, const Batch<MAXB>& b, TmaMaps<MAXB>& maps, float* part,
                                    long long ws_floats, cudaStream_t s) {
    for (int i = 0; i < b.n; ++i) {
        const cudaError_t e = encode_grad_map(g.inst[(size_t)i], &maps.m[i]);
        if (e != cudaSuccess) return e;
    }
    return launch_adjoint_partials_tma(b, maps, part, ws_floats, s, nullptr);
}

static cudaError_t run_group(const Group& g, Op op, bool bf16, float* part, long long ws_floats,
                             cudaStream_t s) {
    (void)cudaGetLastError();  // a launch must not report an earlier call's returned error
    if (g.inst.size() == 1) {
        Batch<1> b;
        to_batch(g, b);
        if (op == Op::Forward) {
            if (bf16_odd_strips(b.inst[0], bf16, g.generic)) b.total_units = b.inst[0].units;
            const int rb = forward_tma_rows(b.inst[0], bf16, g.generic);
            if (rb > 0) {
                CUtensorMap map;
                const cudaError_t e = encode_field_map(b.inst[0], bf16, rb, &map);
                if (e == cudaSuccess) return launch_forward_tma(b, bf16, 3, map, rb, s, nullptr);
            }
            return launch_forward(b, bf16, g.generic, s, nullptr);
        }
        if (op == Op::AdjointPartials) {
            if (g.tma) {
                TmaMaps<1> maps;
                return run_partials_tma(g, b, maps, part, ws_floats, s);
            }
            return launch_adjoint_partials(b, g.generic, part, ws_floats, s, nullptr);
        }
        return launch_adjoint_reduce(b, part, ws_floats, s, nullptr);
    }
    static thread_local Batch<kMaxBatch> b;  // ~9 KB: kept off the stack
    to_batch(g, b);
    if (op == Op::Forward) return launch_forward(b, bf16, g.generic, s, nullptr);
    if (op == Op::AdjointPartials) {
        if (g.tma) {
            static thread_local TmaMaps<kMaxBatch> maps;  // 8 KB
            return run_partials_tma(g, b, maps, part, ws_floats, s);
        }
        return launch_adjoint_partials(b, g.generic, part, ws_floats, s, nullptr);
    }
    return launch_adjoint_reduce(b, part, ws_floats, s, nullptr);
}

static bsi_status check_instances(const bsi_instance* inst, int n, bool fwd, bool adj, bsi_dtype dt) {
    if (n < 0 || (n > 0 && !inst)) return BSI_ERR_BATCH;
    for (int i = 0; i < n; ++i) {
        const bsi_status st = check_geom(&inst[i].geom);
        if (st != BSI_OK) return st;
        const bool empty = empty_volume(inst[i].geom);
        if (fwd && !empty) {
            if (!inst[i].phi || !inst[i].field) return BSI_ERR_NULL;
            if (misaligned(inst[i].phi, 4) || misaligned(inst[i].field, dt == BSI_BF16 ? 2 : 4))
                return BSI_ERR_ALIGN;
        }
        if (adj) {
            if (!inst[i].grad_phi || (!empty && !inst[i].grad_field)) return BSI_ERR_NULL;
            if (misaligned(inst[i].grad_phi, 4) || misaligned(inst[i].grad_field, 4)) return BSI_ERR_ALIGN;
        }
    }
    return BSI_OK;
}

// Instance descriptors; for the adjoint (with the tensor-copy path allowed or
// not, as the launch will run) zchunk comes from choose_zchunk unless the
// tile-config table fixes it.
static std::vector<InstDesc> descs(const bsi_instance* inst, int n, bool adjoint, bool bf16 = false,
                                   bool allow_tma = false, long long max_floats = -1) {
    std::vector<InstDesc> v((size_t)n);
    for (int i = 0; i < n; ++i) {
        InstDesc& d = v[(size_t)i];
        fill_desc(d, inst[i].geom, adjoint, bf16);
        d.phi = inst[i].phi;
        d.field = inst[i].field;
        d.grad = inst[i].grad_field;
        d.dphi = inst[i].grad_phi;
        const bsi_geom& g = inst[i].geom;
        if (adjoint) {
            const bool t = allow_tma && tma_geometry_ok(d);
            const bool fixed = lookup_config(g.dx, g.dy, g.dz).adj_zchunk > 0;
            if (t && two_row_units(d, n)) set_jrows(d, kTmaJrows);
            if (!fixed) set_zchunk(d, choose_zchunk(d, t, max_floats));
            if (d.jrows > 1 && max_floats >= 0 && adj_floats(d) > max_floats) {
                // no plan of two tile-rows per unit fits the fixed scratch: one tile-row
                set_jrows(d, 1);
                if (!fixed) set_zchunk(d, choose_zchunk(d, t, max_floats));
            }
        }
    }
    return v;
}

static bsi_status forward_impl(const bsi_instance* inst, int n, bsi_dtype dt, cudaStream_t s) {
    if (dt != BSI_F32 && dt != BSI_BF16) return BSI_ERR_DTYPE;
    bsi_status st = check_instances(inst, n, true, false, dt);
    if (st != BSI_OK) return st;
    std::vector<InstDesc> all = descs(inst, n, false, dt == BSI_BF16);
    all.erase(std::remove_if(all.begin(), all.end(), [](const InstDesc& d) { return d.units == 0; }), all.end());
    for (const Group& g : plan(all, nullptr)) {
        const cudaError_t e = run_group(g, Op::Forward, dt == BSI_BF16, nullptr, 0, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BSI_OK;
}

// fixed_scratch: ws is the library's no-alloc array; plans are chosen to fit
// it, and only the chosen plan's size is checked.
static bsi_status adjoint_impl(const bsi_instance* inst, int n, void* ws, size_t ws_bytes, cudaStream_t s,
                               bool fixed_scratch = false) {
    bsi_status st = check_instances(inst, n, false, true, BSI_F32);
    if (st != BSI_OK) return st;
    long long ws_floats = 0;
    const bool tma = tensor_map_encoder() != nullptr;
    const std::vector<Group> groups =
        plan(descs(inst, n, true, false, tma, fixed_scratch ? (long long)(ws_bytes / sizeof(float)) : -1),
             &ws_floats, tma);
    // the documented size (the bound over zchunk choices), not only this plan's
    long long bound = 0;
    if (!fixed_scratch)
        for (int i = 0; i < n; ++i) bound += adj_floats_bound(inst[i].geom);
    if ((size_t)std::max(bound, ws_floats) * sizeof(float) > ws_bytes) return BSI_ERR_WORKSPACE;
    if (ws_floats > 0 && !ws) return BSI_ERR_WORKSPACE;
    if (ws && misaligned(ws, 16)) return BSI_ERR_ALIGN;
    float* part = static_cast<float*>(ws);
    for (const Group& g : groups) {
        cudaError_t e = run_group(g, Op::AdjointPartials, false, part, ws_floats, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (const Group& g : groups) {
        cudaError_t e = run_group(g, Op::AdjointReduce, false, part, ws_floats, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BSI_OK;
}

// ----------------------------------------------------------- self-check

struct RangeChecker {
    int bad = 0;
    char msg[256] = "";
    void fail(const char* what, long long a, long long b) {
        if (!bad) std::snprintf(msg, sizeof msg, "%s (%lld, %lld)", what, a, b);
        ++bad;
    }
};

// Checks that slot_unit hands every unit of a launch to exactly one slot, for
// a spread of grid shapes (the actual grid depends on the device), and that
// each slot's units increase (the kernels scan instances forward).
static void check_slots(long long total, RangeChecker& rc) {
    const int ctas_list[] = {1, 3, 152, 304, 1000};
    const int wpc_list[] = {1, 5, 8};
    std::vector<unsigned char> seen((size_t)total, 0);
    for (int spread = 0; spread < 2; ++spread)
    for (int ctas : ctas_list)
        for (int wpc : wpc_list) {
            std::fill(seen.begin(), seen.end(), 0);
            for (int c = 0; c < ctas; ++c)
                for (int w = 0; w < wpc; ++w) {
                    long long prev = -1;
                    for (long long r = 0;; ++r) {
                        const long long u = slot_unit(r, c, w, ctas, wpc, total, spread != 0);
                        if (u < 0) break;
                        if (u >= total || u <= prev) {
                            rc.fail("slot order", u, prev);
                            break;
                        }
                        seen[(size_t)u]++;
                        prev = u;
                    }
                }
            for (long long u = 0; u < total; ++u)
                if (seen[(size_t)u] != 1) {
                    rc.fail("unit not taken exactly once", u, ctas * 100 + wpc);
                    break;
                }
        }
}

// Walks every unit of a forward launch plan and checks, with the kernels' own
// index functions, that each read and write lies inside its buffer, that each
// staging copy fits its shared-memory buffer, and (when `cover` is set) that
// the rows of the units tile the field exactly once.
// ob: staging bytes per voxel (12 / 6 forward FP32 / BF16, 12 for T in both
// resampling modes); outputs are checked as voxel ranges.
// The tensor-store path of a single-volume forward (as run_group plans it for a
// 16-byte-aligned field): every box starts on a 16-byte boundary at a
// non-negative coordinate, is at most 256 elements wide, covers exactly its
// strip (or runs past the volume's end, where the copy clips it), stays in its
// tile-row, and every lane's staging stays in its block row or the spare slot.
static void check_forward_tma(const InstDesc& d0, bool bf16, int c, RangeChecker& rc) {
    InstDesc d = d0;
    if (c == 3) bf16_odd_strips(d, bf16, false);
    if (c == 1 && !bf16 && d.dx == 4) return;   // direct stores (bsi_scalar_forward)
    const int rb = fwd_tma_rows(d.X, d.dx, d.dy, d.gcells, bf16, c);
    if (rb <= 0) return;
    const int es = bf16 ? 2 : 4, tile = d.dx * c * es;
    const int rowb = fwd_tma_row_bytes(d.gcells, d.dx, bf16, c);
    const int blk = pad128(rb * rowb), wsm = fwd_tma_warp_smem(blk);
    if (rowb % 16 != 0 || rowb / 8 > 256) rc.fail("tensor-store box width", rowb, 256 * 8);
    if (d.dy % rb != 0 || rb * rowb > blk) rc.fail("tensor-store block rows", rb, d.dy);
    if (tile > 128) rc.fail("halo lane slot", tile, 128);
    if ((long long)warps_per_cta(wsm, d.warps_req) * wsm + 128 > kSmemBudget)
        rc.fail("tensor-store shared memory over budget", wsm, kSmemBudget);
    if ((long long)c * d.X * es % 16 != 0) rc.fail("tensor-store row pitch", d.X, es);
    for (long long ul = 0; ul < d.units; ++ul) {
        const FwdUnit u = fwd_unit(d, ul);
        const long long xb = (long long)u.x0 * c * es;
        if (xb < 0 || xb % 16 != 0) rc.fail("tensor-store box start", u.x0, xb);
        if (u.x0 + d.gcells * d.dx < d.X && u.nvox != d.gcells * d.dx) rc.fail("box past its strip", u.x0, u.nvox);
        if (u.ncell > d.gcells || (long long)(u.ncell - 1) * tile + tile > rowb) rc.fail("lane past block row", u.ncell, rowb);
    }
}

static void check_forward_group(const Group& g, int ob, RangeChecker& rc, bool cover) {
    const int buf = stage_buf_bytes(g.dxmax);
    for (const InstDesc& d : g.inst) {
        const long long phi_elems = 3LL * d.nx * d.ny * d.nz;
        const long long nvox_all = (long long)d.X * d.Y * d.Z;
        std::vector<unsigned char> hit(cover ? (size_t)d.X * d.Y * d.Z : 0, 0);
        for (long long ul = 0; ul < d.units; ++ul) {
            const FwdUnit u = fwd_unit(d, ul);
            if (u.ncell < 1 || u.nvox < 1) rc.fail("forward unit without tiles", ul, u.ncell);
            for (int lane = 0; lane < kLanes; ++lane) {
                const int col = u.cell0 + lane;
                if (col >= d.nx) continue;
                for (int n = 0; n < 4; ++n)
                    for (int m = 0; m < 4; ++m) {
                        const long long e = phi_elem(d, u.kz + n, u.jy + m, col);
                        if (e < 0 || e + 3 > phi_elems) rc.fail("phi read", e, phi_elems);
                    }
                if (lane < u.ncell && lane * d.dx >= u.nvox) rc.fail("emitting lane past strip", lane, u.nvox);
            }
            const int z0 = u.kz * d.dz, zn = imin(d.dz, d.Z - z0);
            const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
            // a specialised spacing stages all 32 lanes x dx voxels (past the row end too)
            const int staged = d.dx <= kMaxSpecializedDx && !g.generic ? kLanes * d.dx : u.nvox;
            if (u.nvox > staged || 15 + staged * ob > buf) rc.fail("staging overflow", staged, buf);
            if (warps_per_cta(fwd_warp_smem(buf)) * fwd_warp_smem(buf) > kSmemBudget)
                rc.fail("forward shared memory over budget", buf, kSmemBudget);
            for (int rz = 0; rz < zn; ++rz)
                for (int ry = 0; ry < yn; ++ry) {
                    const long long v0 = field_elem(d, z0 + rz, y0 + ry, u.x0) / 3;   // voxel index
                    if (v0 < 0 || v0 + u.nvox > nvox_all) rc.fail("field write", v0, nvox_all);
                    if (cover)
                        for (int x = 0; x < u.nvox; ++x) hit[(size_t)(v0 + x)]++;
                }
        }
        if (cover)
            for (size_t i = 0; i < hit.size(); ++i)
                if (hit[i] != 1) {
                    rc.fail("voxel written != once", (long long)i, hit[i]);
                    break;
                }
    }
}

static void check_adjoint_group(const Group& g, long long ws_floats, RangeChecker& rc, bool cover) {
    const int buf = stage_buf_bytes(g.dxmax);
    std::vector<unsigned char> written(cover ? (size_t)(ws_floats / 3 + 1) : 0, 0);
    for (const InstDesc& d : g.inst) {
        const long long field_elems = 3LL * d.X * d.Y * d.Z;
        for (long long ul = 0; ul < d.units; ++ul) {
            const AdjUnit u = adj_unit(d, ul);
            if (u.kz1 <= u.kz0) rc.fail("adjoint unit without planes", ul, u.kz0);
            if (g.tma) {
                // tensor-copy path: the box fits a stage, holds every float of the
                // unit's cells, and every lane's reads stay inside a box row
                const int tsb = g.tma_stage, rb = d.tma_rows;
                const int nb = tma_boxes(d.dx), W = tma_box_width(d.dx);
                if (!tma_geometry_ok(d) || d.dx > g.dxmax) rc.fail("tensor-copy group member", d.dx, d.dy);
                if (rb < 1 || rb > kTmaMaxRows || d.dy % rb != 0) rc.fail("rows per block", rb, d.dy);
                if (W > 256 || (8 * W) % 16 != 0) rc.fail("box width", W, 256);
                if (tma_block_bytes(d.dx, rb) > tsb || tsb % 128 != 0) rc.fail("block over stage", rb, tsb);
                const int f0 = tma_first_float(u, d.dx), gx0 = tma_group_of(f0), shift = f0 - 4 * gx0;
                if (shift < 0 || shift > 3 || 4LL * gx0 > f0) rc.fail("box start", f0, gx0);
                // every lane's dx voxels lie inside a row of its box (box bx covers the
                // floats [4 gx0 + 48 dx bx, + 2 W), lanes 16 bx .. of it)
                for (int lane = 0; lane < kLanes; ++lane) {
                    const int bx = nb == 1 ? 0 : lane / 16;
                    const int rel = shift + 3 * d.dx * (lane - 16 * bx);   // floats from the box start
                    if (rel < 0 || rel + 3 * d.dx > 2 * W) rc.fail("lane reads past box row", lane, rel);
                    const long long abs0 = 4LL * gx0 + 48LL * d.dx * bx + rel;
                    if (abs0 != 3LL * d.dx * (u.col0 - kHalo + lane)) rc.fail("lane box offset", lane, abs0);
                }
                const int st = tma_default_stages(tsb);
                const int w = tma_warps_per_cta(tsb, st, 0, d.jrows);
                if (st < kTmaMinStages || st > kTmaMaxStages || (long long)w * tma_warp_smem(tsb, st) + 128 > kTmaSmemBudget)
                    rc.fail("tensor-copy shared memory over budget", w, tsb);
            }
            // a bulk load covers the 16-byte-aligned superset of the row: <= nbytes + 30
            if (!g.tma && 30 + u.nvox * 12 > buf) rc.fail("staging overflow", u.nvox, buf);
            // unpredicated reads of a specialised spacing: every lane reads dx voxels,
            // inside [0, nvox) or, in a ragged unit, the zeros [nvox, nvox + zv)
            const bool spec = d.dx <= kMaxSpecializedDx && !g.generic && !g.tma;
            bool ragged = false;
            for (int lane = 0; lane < kLanes; ++lane) {
                const int cell = u.col0 - kHalo + lane;
                const int nv = (cell >= 0 && cell < d.ncx) ? imin(d.dx, d.X - cell * d.dx) : 0;
                ragged = ragged || nv != d.dx;
            }
            const int zv = imin(d.dx, kLanes * d.dx - u.nvox);
            if (spec && ragged && 15 + 12 * (u.nvox + zv) > buf) rc.fail("zeroed tail overflow", u.nvox + zv, buf);
            if (!g.tma && warps_per_cta(adj_warp_smem(buf)) * adj_warp_smem(buf) > kSmemBudget)
                rc.fail("adjoint shared memory over budget", buf, kSmemBudget);
            for (int lane = 0; lane < kLanes; ++lane) {
                const int cell = u.col0 - kHalo + lane;
                const int nv = (cell >= 0 && cell < d.ncx) ? imin(d.dx, d.X - cell * d.dx) : 0;
                const int xl = cell * d.dx - u.xs;
                if (nv > 0 && (xl < 0 || xl + nv > u.nvox)) rc.fail("lane voxels outside strip", xl, u.nvox);
                if (spec) {
                    const int rl = nv == 0 ? u.nvox : xl;   // the kernel's read start
                    if (rl < 0 || rl + d.dx > (ragged ? u.nvox + zv : u.nvox))
                        rc.fail("unpredicated read outside row and zeros", rl, u.nvox);
                    if (nv > 0 && nv < d.dx && xl + nv != u.nvox)   // its missing voxels are the zeros
                        rc.fail("cut tile does not end at the row end", xl + nv, u.nvox);
                }
                const int j = lane - kHalo;
                if (j < 0 || u.col0 + j >= d.nx) continue;
                for (int pz = 0; pz < u.kz1 - u.kz0 + kHalo; ++pz)
                    for (int m = 0; m < d.jrows + kHalo; ++m) {
                        const long long e = part_elem(d, ul, pz, m, j);
                        if (e < 0 || e + 3 > ws_floats) rc.fail("partial write", e, ws_floats);
                        else if (cover) written[(size_t)(e / 3)] = 1;
                    }
            }
            for (int kz = u.kz0; kz < u.kz1; ++kz) {
                const int z0 = kz * d.dz, zn = imin(d.dz, d.Z - z0);
                const int y0 = u.jy * d.dy, yn = imin(d.jrows * d.dy, d.Y - y0);
                for (int rz = 0; rz < zn; ++rz)
                    for (int ry = 0; ry < yn; ++ry) {
                        const long long e0 = field_elem(d, z0 + rz, y0 + ry, u.xs);
                        if (e0 < 0 || e0 + 3LL * u.nvox > field_elems) rc.fail("grad read", e0, field_elems);
                    }
            }
        }
    }
    // the reduce: every partial read lies in the workspace and was written by phase 1
    for (const InstDesc& d : g.inst) {
        for (int gz = 0; gz < d.nz; ++gz)
            for (int gy = 0; gy < d.ny; ++gy)
                for (int gx = 0; gx < d.nx; ++gx) {
                    if (d.nzc <= 0) continue;
                    const int xg = gx / kGroupCells, j = gx - xg * kGroupCells;
                    const int zc_hi = imin(d.nzc - 1, gz / d.zchunk);
                    const int zc_lo =
                        gz - d.zchunk - kHalo + 1 > 0 ? (int)cdiv(gz - d.zchunk - kHalo + 1, d.zchunk) : 0;
                    for (int zc = zc_lo; zc <= zc_hi; ++zc) {
                        const int pz = gz - zc * d.zchunk;
                        const int planes = imin(d.zchunk, d.ncz - zc * d.zchunk) + kHalo;
                        if (pz >= planes) continue;
                        // the units whose tile-rows reach grid row gy, as the reduce finds them
                        const int uy0 = gy / d.jrows, m0 = gy - uy0 * d.jrows;
                        for (int q = 0; q < 4; ++q) {
                            const int uy = uy0 - q, m = m0 + q * d.jrows;
                            if (uy < 0 || uy >= d.ncyu || m >= d.jrows + kHalo) continue;
                            const long long ul = ((long long)zc * d.ncyu + uy) * d.nxg + xg;
                            const long long e = part_elem(d, ul, pz, m, j);
                            if (e < 0 || e + 3 > ws_floats) rc.fail("partial read", e, ws_floats);
                            else if (cover && !written[(size_t)(e / 3)]) rc.fail("partial read before write", e, gx);
                        }
                    }
                }
    }
}

// ----------------------------------------------------------- resampling

static bsi_status check_floating(int64_t fX, int64_t fY, int64_t fZ, const float* floating) {
    if (fX < 1 || fY < 1 || fZ < 1 || fX > BSI_MAX_DIM || fY > BSI_MAX_DIM || fZ > BSI_MAX_DIM) return BSI_ERR_DIMS;
    if (fX * fY > (int64_t)BSI_MAX_FLOATING_ELEMS / fZ) return BSI_ERR_DIMS;   // 32-bit element offsets
    if (!floating) return BSI_ERR_NULL;
    if (misaligned(floating, 4)) return BSI_ERR_ALIGN;
    return BSI_OK;
}

// One resampling launch (value or gradient mode) over the forward's units.
static bsi_status run_resample(const bsi_geom* g, const float* phi, const float* floating, int64_t fX, int64_t fY,
                               int64_t fZ, const float* grad_warped, void* out, bool grad, cudaStream_t s) {
    InstDesc d;
    fill_desc(d, *g, false, false);
    if (d.units == 0) return BSI_OK;
    d.phi = phi;
    d.field = out;
    d.image = floating;
    d.gwarp = grad_warped;
    d.fX = (int)fX;
    d.fY = (int)fY;
    d.fZ = (int)fZ;
    Group grp;
    grp.generic = d.dx > kMaxSpecializedDx;
    grp.dxmax = d.dx;
    grp.warps_req = d.warps_req;
    grp.inst.push_back(d);
    Batch<1> b;
    to_batch(grp, b);
    (void)cudaGetLastError();
    const cudaError_t e = launch_resample(b, grad, grp.generic, s, nullptr);
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

static size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// Strip width of the scalar forward: a row of 4-byte (FP32) voxels starts on a
// 16-byte boundary when x0 and X are multiples of 4 -- the rule of the 3-channel
// field (12-byte voxels) -- so fwd_strip_tiles applies unchanged.

}  // namespace bsi

using namespace bsi;

extern "C" {

bsi_status bsi_geom_rational_init(bsi_geom_rational* g, int64_t X, int64_t Y, int64_t Z, const int32_t num[3],
                                  const int32_t den[3], const int32_t off[3]) {
    if (!g || !num || !den || !off) return BSI_ERR_NULL;
    std::memset(g, 0, sizeof *g);
    g->X = X;
    g->Y = Y;
    g->Z = Z;
    for (int a = 0; a < 3; ++a) {
        g->num[a] = num[a];
        g->den[a] = den[a];
        g->off[a] = off[a];
    }
    if (X < 0 || Y < 0 || Z < 0 || X > BSI_MAX_DIM || Y > BSI_MAX_DIM || Z > BSI_MAX_DIM) return BSI_ERR_DIMS;
    for (int a = 0; a < 3; ++a)
        if (den[a] < 1 || den[a] > BSI_MAX_RATIONAL_DEN || num[a] < den[a] || num[a] > BSI_MAX_SPACING * den[a] ||
            off[a] < 0 || off[a] >= num[a])
            return BSI_ERR_SPACING;
    g->nx = rational_dim(X, num[0], den[0], off[0]);
    g->ny = rational_dim(Y, num[1], den[1], off[1]);
    g->nz = rational_dim(Z, num[2], den[2], off[2]);
    return BSI_OK;
}

bsi_status bsi_geom_init(bsi_geom* g, int64_t X, int64_t Y, int64_t Z, int32_t dx, int32_t dy, int32_t dz) {
    if (!g) return BSI_ERR_NULL;
    std::memset(g, 0, sizeof *g);
    g->X = X;
    g->Y = Y;
    g->Z = Z;
    g->dx = dx;
    g->dy = dy;
    g->dz = dz;
    if (X < 0 || Y < 0 || Z < 0 || X > BSI_MAX_DIM || Y > BSI_MAX_DIM || Z > BSI_MAX_DIM) return BSI_ERR_DIMS;
    if (dx < 1 || dy < 1 || dz < 1 || dx > BSI_MAX_SPACING || dy > BSI_MAX_SPACING || dz > BSI_MAX_SPACING)
        return BSI_ERR_SPACING;
    g->nx = cdiv(X, dx) + 3;
    g->ny = cdiv(Y, dy) + 3;
    g->nz = cdiv(Z, dz) + 3;
    return BSI_OK;
}

bsi_status bsi_field_forward(const bsi_geom* g, const float* phi, void* field, bsi_dtype out_dtype,
                             bsi_stream_t stream) {
    if (!g) return BSI_ERR_NULL;
    bsi_instance in;
    std::memset(&in, 0, sizeof in);
    in.geom = *g;
    in.phi = phi;
    in.field = field;
    return forward_impl(&in, 1, out_dtype, reinterpret_cast<cudaStream_t>(stream));
}

size_t bsi_adjoint_workspace_bytes(const bsi_geom* g) {
    if (check_geom(g) != BSI_OK) return 0;
    return (size_t)adj_floats_bound(*g) * sizeof(float);
}

bsi_status bsi_field_adjoint(const bsi_geom* g, const float* grad_field, float* grad_phi, void* workspace,
                             size_t workspace_bytes, bsi_stream_t stream) {
    if (!g) return BSI_ERR_NULL;
    bsi_instance in;
    std::memset(&in, 0, sizeof in);
    in.geom = *g;
    in.grad_field = grad_field;
    in.grad_phi = grad_phi;
    return adjoint_impl(&in, 1, workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

bsi_status bsi_field_forward_batched(const bsi_instance* inst, int n, bsi_dtype out_dtype, bsi_stream_t stream) {
    return forward_impl(inst, n, out_dtype, reinterpret_cast<cudaStream_t>(stream));
}

size_t bsi_batched_adjoint_workspace_bytes(const bsi_instance* inst, int n) {
    if (n < 0 || (n > 0 && !inst)) return 0;
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        if (check_geom(&inst[i].geom) != BSI_OK) return 0;
        total += adj_floats_bound(inst[i].geom);
    }
    return (size_t)total * sizeof(float);
}

bsi_status bsi_field_adjoint_batched(const bsi_instance* inst, int n, void* workspace, size_t workspace_bytes,
                                     bsi_stream_t stream) {
    return adjoint_impl(inst, n, workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

const char* bsi_status_string(bsi_status s) {
    switch (s) {
        case BSI_OK: return "BSI_OK";
        case BSI_ERR_NULL: return "BSI_ERR_NULL: a required pointer is NULL";
        case BSI_ERR_DIMS: return "BSI_ERR_DIMS: volume dimension out of range";
        case BSI_ERR_SPACING: return "BSI_ERR_SPACING: spacing outside 1..64";
        case BSI_ERR_GRID_MISMATCH: return "BSI_ERR_GRID_MISMATCH: grid dims differ from ceil(N/d)+3";
        case BSI_ERR_DTYPE: return "BSI_ERR_DTYPE: unknown output dtype";
        case BSI_ERR_ALIGN: return "BSI_ERR_ALIGN: pointer not naturally aligned";
        case BSI_ERR_WORKSPACE: return "BSI_ERR_WORKSPACE: workspace missing or too small";
        case BSI_ERR_CUDA: return "BSI_ERR_CUDA: a CUDA call failed";
        case BSI_ERR_DEVICE_STATUS: return "BSI_ERR_DEVICE_STATUS: a kernel recorded an error";
        case BSI_ERR_BATCH: return "BSI_ERR_BATCH: bad instance count or list";
        case BSI_ERR_SCRATCH_LIMIT: return "BSI_ERR_SCRATCH_LIMIT: volume needs more than the built-in 64 MiB scratch";
    }
    return "unknown bsi_status";
}

const char* bsi_last_cuda_error(void) { return t_cuda_msg; }

bsi_status bsi_set_tile_configs(const bsi_tile_config* cfgs, int n) {
    if (n < 0 || n > BSI_MAX_TILE_CONFIGS || (n > 0 && !cfgs)) return BSI_ERR_BATCH;
    for (int i = 0; i < n; ++i)
        if (!config_valid(cfgs[i])) return BSI_ERR_SPACING;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg.assign(cfgs, cfgs + n);
    return BSI_OK;
}

bsi_status bsi_get_tile_config(int32_t dx, int32_t dy, int32_t dz, bsi_tile_config* out) {
    if (!out) return BSI_ERR_NULL;
    if (dx < 1 || dy < 1 || dz < 1 || dx > BSI_MAX_SPACING || dy > BSI_MAX_SPACING || dz > BSI_MAX_SPACING)
        return BSI_ERR_SPACING;
    bsi_tile_config c = lookup_config(dx, dy, dz);
    c.dx = dx;
    c.dy = dy;
    c.dz = dz;
    if (c.adj_warps == 0) c.adj_warps = kAdjWarpsMax;
    if (c.fwd_warps == 0) c.fwd_warps = kMaxWarpsPerCta;
    // fwd_strip_tiles stays 0 when unset: it then depends on the volume (X % 4) and dtype
    *out = c;
    return BSI_OK;
}

bsi_status bsi_check_device_status(bsi_stream_t stream, uint32_t* flags) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    static thread_local unsigned words[5];
    cudaError_t e = forward_err_read_clear(&words[0], s);
    if (e == cudaSuccess) e = adjoint_err_read_clear(&words[1], s);
    if (e == cudaSuccess) e = resample_err_read_clear(&words[2], s);
    if (e == cudaSuccess) e = variants_err_read_clear(&words[3], s);
    if (e == cudaSuccess) e = rational_err_read_clear(&words[4], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint32_t w = words[0] | words[1] | words[2] | words[3] | words[4];
    if (flags) *flags = w;
    return w ? BSI_ERR_DEVICE_STATUS : BSI_OK;
}

// Scalar interpolation takes the tensor-store path where fwd_tma_rows allows it,
// except FP32 at x-spacing 4, whose lanes store their 16-byte tiles directly
// (4x zoom to 512 x 512 x 300: 0.070 ms direct, 0.078 ms in blocks; blocks at
// spacing 3: 0.157 -> 0.140 ms, BF16 at 4: 0.107 -> 0.096 ms).
constexpr bool kScalarTma = true;

bsi_status bsi_scalar_forward(const bsi_geom* g, const float* coeff, void* out, bsi_dtype out_dtype,
                              bsi_stream_t stream) {
    bsi_status st = check_geom(g);
    if (st != BSI_OK) return st;
    if (out_dtype != BSI_F32 && out_dtype != BSI_BF16) return BSI_ERR_DTYPE;
    if (empty_volume(*g)) return BSI_OK;
    if (!coeff || !out) return BSI_ERR_NULL;
    if (misaligned(coeff, 4) || misaligned(out, out_dtype == BSI_BF16 ? 2 : 4)) return BSI_ERR_ALIGN;
    InstDesc d;
    fill_desc(d, *g, false, out_dtype == BSI_BF16);
    d.phi = coeff;
    d.field = out;
    Group grp;
    grp.generic = d.dx > kMaxSpecializedDx;
    grp.dxmax = d.dx;
    grp.warps_req = d.warps_req;
    grp.inst.push_back(d);
    Batch<1> b;
    to_batch(grp, b);
    (void)cudaGetLastError();
    const bool bf16 = out_dtype == BSI_BF16;
    const int rb = kScalarTma && (bf16 || b.inst[0].dx != 4) ? forward_tma_rows(b.inst[0], bf16, grp.generic, 1) : 0;
    if (rb > 0) {
        CUtensorMap map;
        if (encode_field_map(b.inst[0], bf16, rb, &map, 1) == cudaSuccess) {
            const cudaError_t e = launch_forward_tma(b, bf16, 1, map, rb, reinterpret_cast<cudaStream_t>(stream), nullptr);
            return e == cudaSuccess ? BSI_OK : cuda_fail(e);
        }
    }
    const cudaError_t e = launch_forward_scalar(b, bf16, grp.generic, reinterpret_cast<cudaStream_t>(stream), nullptr);
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

bsi_status bsi_field_forward_variant(const bsi_geom* g, const float* phi, float* field, int32_t variant,
                                     bsi_stream_t stream) {
    if (variant == BSI_VARIANT_SEPARABLE) return bsi_field_forward(g, phi, field, BSI_F32, stream);
    if (variant != BSI_VARIANT_TT && variant != BSI_VARIANT_TTLI) return BSI_ERR_DTYPE;
    bsi_status st = check_geom(g);
    if (st != BSI_OK) return st;
    if (g->dx > 32 || g->dy > 32 || g->dz > 32) return BSI_ERR_SPACING;
    if (empty_volume(*g)) return BSI_OK;
    if (!phi || !field) return BSI_ERR_NULL;
    if (misaligned(phi, 4) || misaligned(field, 4)) return BSI_ERR_ALIGN;
    InstDesc d;
    fill_desc(d, *g, false, false);
    d.phi = phi;
    d.field = field;
    Group grp;
    grp.dxmax = d.dx;
    grp.inst.push_back(d);
    Batch<1> b;
    to_batch(grp, b);
    (void)cudaGetLastError();
    const cudaError_t e = launch_forward_tile_variant(b, variant == BSI_VARIANT_TTLI,
                                                      reinterpret_cast<cudaStream_t>(stream), nullptr);
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

static bsi_status check_rational(const bsi_geom_rational* g) {
    if (!g) return BSI_ERR_NULL;
    if (g->X < 0 || g->Y < 0 || g->Z < 0 || g->X > BSI_MAX_DIM || g->Y > BSI_MAX_DIM || g->Z > BSI_MAX_DIM)
        return BSI_ERR_DIMS;
    for (int a = 0; a < 3; ++a) {
        const int32_t n = g->num[a], d = g->den[a], o = g->off[a];
        if (d < 1 || d > BSI_MAX_RATIONAL_DEN || n < d || n > BSI_MAX_SPACING * d || o < 0 || o >= n)
            return BSI_ERR_SPACING;
    }
    if (g->nx != rational_dim(g->X, g->num[0], g->den[0], g->off[0]) ||
        g->ny != rational_dim(g->Y, g->num[1], g->den[1], g->off[1]) ||
        g->nz != rational_dim(g->Z, g->num[2], g->den[2], g->off[2]))
        return BSI_ERR_GRID_MISMATCH;
    if (g->nx > BSI_MAX_RATIONAL_NX) return BSI_ERR_DIMS;
    return BSI_OK;
}

static RatDesc rat_desc(const bsi_geom_rational& g) {
    RatDesc d;
    std::memset(&d, 0, sizeof d);
    d.X = (int)g.X;
    d.Y = (int)g.Y;
    d.Z = (int)g.Z;
    for (int a = 0; a < 3; ++a) {
        d.num[a] = g.num[a];
        d.den[a] = g.den[a];
        d.off[a] = g.off[a];
    }
    d.nx = (int)g.nx;
    d.ny = (int)g.ny;
    d.nz = (int)g.nz;
    return d;
}

bsi_status bsi_field_forward_rational(const bsi_geom_rational* g, const float* phi, float* field,
                                      bsi_stream_t stream) {
    bsi_status st = check_rational(g);
    if (st != BSI_OK) return st;
    if (g->X == 0 || g->Y == 0 || g->Z == 0) return BSI_OK;
    if (!phi || !field) return BSI_ERR_NULL;
    if (misaligned(phi, 4) || misaligned(field, 4)) return BSI_ERR_ALIGN;
    RatDesc d = rat_desc(*g);
    d.phi = phi;
    d.field = field;
    (void)cudaGetLastError();
    const cudaError_t e = launch_forward_rational(d, reinterpret_cast<cudaStream_t>(stream), nullptr);
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

size_t bsi_rational_adjoint_workspace_bytes(const bsi_geom_rational* g) {
    if (check_rational(g) != BSI_OK || g->X == 0 || g->Y == 0 || g->Z == 0) return 0;
    return (size_t)rational_adjoint_plan(rat_desc(*g)).part_floats * sizeof(float);
}

bsi_status bsi_field_adjoint_rational(const bsi_geom_rational* g, const float* grad_field, float* grad_phi,
                                      void* workspace, size_t workspace_bytes, bsi_stream_t stream) {
    bsi_status st = check_rational(g);
    if (st != BSI_OK) return st;
    if (!grad_phi) return BSI_ERR_NULL;
    if (misaligned(grad_phi, 4)) return BSI_ERR_ALIGN;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (g->X == 0 || g->Y == 0 || g->Z == 0) {   // no voxel: the gradient is zero
        (void)cudaGetLastError();
        const cudaError_t e = cudaMemsetAsync(grad_phi, 0, (size_t)(g->nx * g->ny * g->nz) * 3 * sizeof(float), s);
        return e == cudaSuccess ? BSI_OK : cuda_fail(e);
    }
    if (!grad_field) return BSI_ERR_NULL;
    if (misaligned(grad_field, 4)) return BSI_ERR_ALIGN;
    const RatDesc d = rat_desc(*g);
    const size_t need = (size_t)rational_adjoint_plan(d).part_floats * sizeof(float);
    if (!workspace || workspace_bytes < need) return BSI_ERR_WORKSPACE;
    if (misaligned(workspace, 16)) return BSI_ERR_ALIGN;
    (void)cudaGetLastError();
    const cudaError_t e = launch_adjoint_rational(d, grad_field, grad_phi, static_cast<float*>(workspace), s);
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

bsi_status bsi_resample_forward(const bsi_geom* g, const float* phi, const float* floating, int64_t fX, int64_t fY,
                                int64_t fZ, float* warped, bsi_stream_t stream) {
    bsi_status st = check_geom(g);
    if (st != BSI_OK) return st;
    if ((st = check_floating(fX, fY, fZ, floating)) != BSI_OK) return st;
    if (empty_volume(*g)) return BSI_OK;
    if (!phi || !warped) return BSI_ERR_NULL;
    if (misaligned(phi, 4) || misaligned(warped, 4)) return BSI_ERR_ALIGN;
    return run_resample(g, phi, floating, fX, fY, fZ, nullptr, warped, false, reinterpret_cast<cudaStream_t>(stream));
}

size_t bsi_resample_backward_workspace_bytes(const bsi_geom* g) {
    if (check_geom(g) != BSI_OK || empty_volume(*g)) return 0;
    return round256((size_t)12 * g->X * g->Y * g->Z) + (size_t)adj_floats_bound(*g) * sizeof(float);
}

bsi_status bsi_resample_backward(const bsi_geom* g, const float* phi, const float* floating, int64_t fX, int64_t fY,
                                 int64_t fZ, const float* grad_warped, float* grad_phi, void* workspace,
                                 size_t workspace_bytes, bsi_stream_t stream) {
    bsi_status st = check_geom(g);
    if (st != BSI_OK) return st;
    if ((st = check_floating(fX, fY, fZ, floating)) != BSI_OK) return st;
    if (!grad_phi) return BSI_ERR_NULL;
    if (misaligned(grad_phi, 4)) return BSI_ERR_ALIGN;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bsi_instance in;
    std::memset(&in, 0, sizeof in);
    in.geom = *g;
    in.grad_phi = grad_phi;
    if (empty_volume(*g)) return adjoint_impl(&in, 1, nullptr, 0, s);   // grad_phi = 0
    if (!phi || !grad_warped) return BSI_ERR_NULL;
    if (misaligned(phi, 4) || misaligned(grad_warped, 4)) return BSI_ERR_ALIGN;
    if (!workspace || workspace_bytes < bsi_resample_backward_workspace_bytes(g)) return BSI_ERR_WORKSPACE;
    if (misaligned(workspace, 16)) return BSI_ERR_ALIGN;
    // G = dL/dwarped * grad F~(x + T(x)) into the workspace, then the adjoint of G
    float* G = static_cast<float*>(workspace);
    const size_t goff = round256((size_t)12 * g->X * g->Y * g->Z);
    st = run_resample(g, phi, floating, fX, fY, fZ, grad_warped, G, true, s);
    if (st != BSI_OK) return st;
    in.grad_field = G;
    return adjoint_impl(&in, 1, static_cast<unsigned char*>(workspace) + goff, workspace_bytes - goff, s);
}

bsi_status bsi_selftest_lost_copy(bsi_stream_t stream) {
    (void)cudaGetLastError();
    const cudaError_t e = launch_selftest_lost_copy(reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BSI_OK : cuda_fail(e);
}

int bsi_version(void) { return 100; }

// Host-only: plans the launches of a batched call exactly as the entry points
// do and checks every global and shared-memory range the kernels will touch
// (see RangeChecker).  op: 0 forward F32, 1 forward BF16, 2 adjoint, 3 / 4
// resampling value / gradient mode (the forward's walk), 5 / 6 scalar forward
// F32 / BF16.  With
// cover != 0 it also checks that forward rows tile each field exactly once and
// that the reduce reads only partials phase 1 writes (memory ~ field size).
// Returns the number of violations; the first is described in msg.
int bsi_selfcheck_ranges(const bsi_instance* inst, int n, int op, int cover, char* msg, size_t msg_len) {
    RangeChecker rc;
    if (n < 0 || (n > 0 && !inst) || op < 0 || op > 6) {
        rc.fail("bad arguments", n, op);
    } else {
        bool ok = true;
        for (int i = 0; i < n; ++i) ok = ok && check_geom(&inst[i].geom) == BSI_OK;
        if (!ok) {
            rc.fail("invalid geometry", n, 0);
        } else if (op != 2) {
            std::vector<InstDesc> all = descs(inst, n, false, op == 1 || op == 6);
            all.erase(std::remove_if(all.begin(), all.end(), [](const InstDesc& d) { return d.units == 0; }),
                      all.end());
            for (const Group& g : plan(all, nullptr)) {
                // staging bytes per voxel: the field (12 FP32, 6 BF16), T for both
                // resampling modes (12), the scalar forward (4 FP32, 2 BF16)
                check_forward_group(g, op == 1 ? 6 : op == 5 ? 4 : op == 6 ? 2 : 12, rc, cover != 0);
                // the single-volume forward's tensor-store path (3 or 1 channels)
                if ((op == 0 || op == 1 || op == 5 || op == 6) && n == 1 && g.inst.size() == 1 && !g.generic)
                    check_forward_tma(g.inst[0], op == 1 || op == 6, op >= 5 ? 1 : 3, rc);
                long long total = 0;
                for (const InstDesc& d : g.inst) total += d.units;
                if (cover) check_slots(total, rc);
            }
        } else {
            long long ws = 0;
            const std::vector<Group> groups = plan(descs(inst, n, true, false, true), &ws, true);
            // the documented workspace (the bound over every plan) holds the planned one
            long long bound = 0;
            for (int i = 0; i < n; ++i) bound += adj_floats_bound(inst[i].geom);
            if (ws > bound) rc.fail("planned workspace over the documented bound", ws, bound);
            // and so does the least bound the no-alloc entry point admits a volume by
            if (n == 1) {
                long long ws1 = 0;
                const long long least = adj_floats_bound(inst[0].geom, true);
                (void)plan(descs(inst, 1, true, false, true, least), &ws1, true);
                if (ws1 > least) rc.fail("no plan fits the least bound", ws1, least);
            }
            for (const Group& g : groups) {
                check_adjoint_group(g, ws, rc, cover != 0);
                long long total = 0;
                for (const InstDesc& d : g.inst) total += d.units;
                if (cover) check_slots(total, rc);
            }
        }
    }
    if (msg && msg_len) {
        std::strncpy(msg, rc.msg, msg_len - 1);
        msg[msg_len - 1] = 0;
    }
    return rc.bad;
}

}  // extern "C"

// ----------------------------------------------------------- adjoint without caller scratch
//
// For callers that cannot allocate device memory (stream capture in progress,
// host applications that own all device allocations, plain C callers without a
// device allocator): the partial sums of bsi_field_adjoint live in a fixed
// array inside the library instead of a caller workspace.

namespace bsi {

constexpr size_t kNoAllocScratchBytes = BSI_NOALLOC_SCRATCH_BYTES;

// In host code this name is only a handle for the runtime; kernels get the
// device address that noalloc_scratch() looks up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  Outside stream
// capture it is looked up afresh on every call (cheap, and right again after a
// cudaDeviceReset has reloaded the module) and remembered per device; during
// capture the remembered address is used, so a first call per device must come
// before any capture (BSI_ERR_CUDA otherwise).
static cudaError_t noalloc_scratch(cudaStream_t s, void** out) {
    static std::mutex mu;
    static std::unordered_map<int, void*> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    auto it = addr.find(dev);
    if (it == addr.end()) return cudaErrorStreamCaptureUnsupported;
    *out = it->second;
    return cudaSuccess;
}

}  // namespace bsi

extern "C" bsi_status bsi_field_adjoint_noalloc(const bsi_geom* g, const float* grad_field, float* grad_phi,
                                                bsi_stream_t stream) {
    if (!g) return BSI_ERR_NULL;
    bsi_instance in;
    std::memset(&in, 0, sizeof in);
    in.geom = *g;
    in.grad_field = grad_field;
    in.grad_phi = grad_phi;
    const bsi_status st = check_instances(&in, 1, false, true, BSI_F32);
    if (st != BSI_OK) return st;
    // the smallest plan must fit; adjoint_impl then picks among the plans that do
    const size_t need = empty_volume(*g) ? 0 : (size_t)adj_floats_bound(*g, true) * sizeof(float);
    if (need > kNoAllocScratchBytes) return BSI_ERR_SCRATCH_LIMIT;
    void* scratch = nullptr;
    if (need > 0) {
        const cudaError_t e = noalloc_scratch(reinterpret_cast<cudaStream_t>(stream), &scratch);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return adjoint_impl(&in, 1, scratch, kNoAllocScratchBytes, reinterpret_cast<cudaStream_t>(stream), true);
}
