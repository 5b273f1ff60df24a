/*
 * bsi.h -- C ABI of the GB300 (sm_103a) cubic B-spline interpolation library.
 *
 * The library turns a free-form-deformation control grid into the dense
 * 3-channel displacement field of a volume (the "BSI transformation" of
 * Eq. 1, Sec. 2.1 of Zachariadis et al., "Accelerating B-spline Interpolation
 * on GPUs: Application to Medical Image Registration"), and applies the
 * transpose of that map to a voxel gradient (the gather of dL/du back onto the
 * control points that every gradient step of the registration loop needs).
 *
 * Definitions shared by every call
 * --------------------------------
 *   Volume X x Y x Z voxels, integer voxel coordinates, x fastest.
 *   Spacing dx, dy, dz: control-point spacing in voxels (Sec. 2.1), 1..64.
 *   Control grid nx x ny x nz with nx = ceil(X/dx) + 3 (likewise ny, nz):
 *   the paper's neighbourhood index i = floor(x/dx) - 1 is stored at column
 *   i + 1, so the grid carries one border point below and two above and
 *   every 4x4x4 neighbourhood is in range.
 *   B_0..B_3 are the uniform cubic B-spline blending functions.
 *
 *   field[z][y][x][c] = sum_{l,m,n=0..3} B_l(u) B_m(v) B_n(w)
 *                         phi[fz+n][fy+m][fx+l][c]
 *   fx = floor(x/dx), u = x/dx - fx   (likewise fy, v and fz, w), c = 0,1,2.
 *
 * Layouts (all row-major, channel-last, channel order x, y, z):
 *   phi, grad_phi      float [nz][ny][nx][3]          (FP32)
 *   field, grad_field  [Z][Y][X][3], FP32 or BF16 field, FP32 grad_field
 *
 * Conventions
 * -----------
 *   - Every buffer is device memory owned by the caller.  The library never
 *     allocates, frees or synchronises inside these calls, so every call may
 *     be captured in a CUDA graph; work is enqueued on `stream`.
 *   - Arguments are validated on the host before anything is enqueued; a
 *     non-BSI_OK return means nothing was launched.  A CUDA launch failure is
 *     BSI_ERR_CUDA (see bsi_last_cuda_error()).  No call aborts or throws.
 *   - Pointers need natural alignment only (4 bytes for FP32 arrays, 2 for a
 *     BF16 field); any such base address is accepted.
 *   - Results are deterministic: the adjoint sums its partials in a fixed
 *     order and uses no atomics.
 */
#ifndef BSI_H
#define BSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* bsi_stream_t;

typedef enum {
    BSI_OK = 0,
    BSI_ERR_NULL = 1,          /* a required pointer is NULL */
    BSI_ERR_DIMS = 2,          /* X, Y or Z negative or above BSI_MAX_DIM */
    BSI_ERR_SPACING = 3,       /* dx, dy or dz outside 1..BSI_MAX_SPACING */
    BSI_ERR_GRID_MISMATCH = 4, /* geom.nx/ny/nz differ from ceil(X/dx)+3 ... */
    BSI_ERR_DTYPE = 5,         /* unknown bsi_dtype */
    BSI_ERR_ALIGN = 6,         /* pointer not naturally aligned */
    BSI_ERR_WORKSPACE = 7,     /* workspace NULL or smaller than required */
    BSI_ERR_CUDA = 8,          /* a CUDA runtime call failed */
    BSI_ERR_DEVICE_STATUS = 9, /* a kernel recorded an error (bsi_check_device_status) */
    BSI_ERR_BATCH = 10,        /* n < 0, or instances == NULL with n > 0 */
    BSI_ERR_SCRATCH_LIMIT = 11 /* volume needs more than BSI_NOALLOC_SCRATCH_BYTES of scratch */
} bsi_status;

typedef enum { BSI_F32 = 0, BSI_BF16 = 1 } bsi_dtype;

#define BSI_MAX_SPACING 64
#define BSI_MAX_DIM (1 << 20)

/* Geometry of one volume and its control grid.  nx, ny, nz state the grid the
 * caller allocated; they must equal ceil(X/dx)+3 etc. (bsi_geom_init fills them). */
typedef struct {
    int64_t X, Y, Z;     /* volume size in voxels, 0..BSI_MAX_DIM each */
    int32_t dx, dy, dz;  /* control-point spacing in voxels, 1..BSI_MAX_SPACING */
    int32_t reserved;    /* set to 0 */
    int64_t nx, ny, nz;  /* control-grid dims */
} bsi_geom;

/* Fills g from the volume size and spacing (grid dims derived).  Returns
 * BSI_ERR_DIMS / BSI_ERR_SPACING for out-of-range values, BSI_ERR_NULL for g==NULL. */
bsi_status bsi_geom_init(bsi_geom* g, int64_t X, int64_t Y, int64_t Z, int32_t dx, int32_t dy,
                         int32_t dz);

/* Forward BSI (Eq. 1, Sec. 2.1): writes the dense field from the control grid.
 *   phi   : device, FP32 [nz][ny][nx][3], read only
 *   field : device, [Z][Y][X][3] of out_dtype (BF16: round to nearest even of
 *           the FP32 result), fully overwritten
 * An empty volume (X, Y or Z == 0) launches nothing and returns BSI_OK. */
bsi_status bsi_field_forward(const bsi_geom* g, const float* phi, void* field, bsi_dtype out_dtype,
                             bsi_stream_t stream);

/* Workspace bytes bsi_field_adjoint needs for geometry g (0 for an empty
 * volume); no counterpart in the paper (its kernels have no adjoint): the
 * most any of its launch plans can use, since the tile-planes (and, on the
 * tensor-copy path, tile-rows) per warp unit are chosen per call (from the
 * device's SM count) unless the tile-config table fixes the tile-planes. */
size_t bsi_adjoint_workspace_bytes(const bsi_geom* g);

/* Adjoint BSI: the transpose of Eq. 1 applied to a voxel gradient,
 *   grad_phi[g][c] = sum over voxels x of W(x, g) * grad_field[x][c],
 * W(x, g) being the Eq. 1 weight of control point g at voxel x.  This is the
 * gradient of any loss L(field) with respect to phi, given dL/dfield.
 *   grad_field : device, FP32 [Z][Y][X][3], read only
 *   grad_phi   : device, FP32 [nz][ny][nx][3], fully overwritten (not accumulated)
 *   workspace  : device scratch of at least bsi_adjoint_workspace_bytes(g)
 *                bytes, 16-byte aligned (BSI_ERR_ALIGN otherwise); contents
 *                on entry are ignored.  May be NULL when the size is 0.
 * Two kernels: per-warp partial sums over tiles, then a fixed-order reduce.
 * A gradient with X % 4 == 0 at a 16-byte-aligned address and dx <= 8 is read
 * by TMA tensor copies (one per block of rows), any other by one bulk copy per
 * row.  With one tile-row per warp unit both add the same terms in the same
 * order (bitwise equal results); on the tensor-copy path a single volume at
 * y-spacing 4..6 takes units of two tile-rows, which sum in another order
 * (equal to rounding).  The same call on the same input always gives the same
 * bits. */
bsi_status bsi_field_adjoint(const bsi_geom* g, const float* grad_field, float* grad_phi,
                             void* workspace, size_t workspace_bytes, bsi_stream_t stream);

/* One volume of a batch.  Unused pointers (field/phi for an adjoint-only call,
 * grad_field/grad_phi for a forward-only call) may be NULL. */
typedef struct {
    bsi_geom geom;
    const float* phi;         /* forward input  FP32 [nz][ny][nx][3] */
    void* field;              /* forward output [Z][Y][X][3], batch out_dtype */
    const float* grad_field;  /* adjoint input  FP32 [Z][Y][X][3] */
    float* grad_phi;          /* adjoint output FP32 [nz][ny][nx][3] */
} bsi_instance;

/* Batched forward over n volumes of uneven size and spacing (a registration
 * batch); no counterpart in the paper, which interpolates one volume per call:
 * Eq. 1 (Sec. 2.1) per instance.  One persistent launch walks the tiles of
 * every volume; instances are
 * passed by value in the kernel parameters (up to 64 per launch, larger
 * batches are split), so no device copy of the descriptors is needed and the
 * call is capturable.  `inst` is host memory, read during the call only. */
bsi_status bsi_field_forward_batched(const bsi_instance* inst, int n, bsi_dtype out_dtype,
                                     bsi_stream_t stream);

/* Workspace bytes bsi_field_adjoint_batched needs for these n instances (no
 * counterpart in the paper): the sum of each instance's bound, 16-byte aligned
 * per instance. */
size_t bsi_batched_adjoint_workspace_bytes(const bsi_instance* inst, int n);

/* Batched adjoint over n volumes (no counterpart in the paper): the transpose
 * of Eq. 1 per instance, as bsi_field_adjoint.  One persistent partial-sum
 * launch over all volumes' tiles, then one reduce launch; grad_phi of every
 * instance is overwritten.  workspace: device, >= the query's bytes, 16-byte
 * aligned; contents on entry ignored. */
bsi_status bsi_field_adjoint_batched(const bsi_instance* inst, int n, void* workspace,
                                     size_t workspace_bytes, bsi_stream_t stream);

/* Adjoint without caller-provided scratch, for callers that cannot allocate
 * device memory: code running while a stream is being captured into a CUDA
 * graph (where cudaMalloc is not allowed), plug-ins that live inside a host
 * application which owns every device allocation through its own pool, and
 * plain C callers that have device buffers for their data but no allocator
 * for temporaries.  The paper has no counterpart; it is an operational
 * variant of bsi_field_adjoint, whose arguments and result it shares.
 *
 * Scratch: a file-scope device array of BSI_NOALLOC_SCRATCH_BYTES (64 MiB)
 * inside the library, held on every device where the library's module is
 * loaded until the process exits.  The call picks tile-planes per warp unit
 * among the plans whose partial sums fit it; a volume that no plan fits is
 * rejected with BSI_ERR_SCRATCH_LIMIT before anything is enqueued (the
 * 512x512x300 volume at spacing 5 needs 44 to 69 MB depending on the plan).
 * The call allocates no device memory: no cudaMalloc, cudaFree or allocating
 * library routine.  A call made while `stream` is not being captured looks up
 * the array's device address (cudaGetSymbolAddress, with the device current)
 * and remembers it per device; a call made during capture uses the remembered
 * address.  So make one call on each device before any stream capture, and
 * after a cudaDeviceReset make one call outside capture again (the reset
 * unloads the module and with it the array).
 * Every call uses the same array, which keeps the previous call's contents.
 * In a normal call the first kernel writes every scratch entry the second
 * one reads, so no clearing is needed.  If a kernel's bounded wait for a bulk
 * copy runs out, the warp that waited stops without writing its entries, and
 * grad_phi may then hold sums that include the previous call's leftovers:
 * bsi_check_device_status reports such a call (BSI_DEVICE_FLAG_TIMEOUT), and its
 * result must not be used.  Calls that overlap on the GPU (different streams,
 * or other threads, without ordering between them) race on the array: order
 * them on one stream or synchronise between them. */
#define BSI_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
bsi_status bsi_field_adjoint_noalloc(const bsi_geom* g, const float* grad_field, float* grad_phi,
                                     bsi_stream_t stream);

/* Launch shape for one spacing class, chosen by the autotuner
 * (paper_2004_05962_gb300/tune.py times candidates and keeps a JSON cache).
 * The paper tunes its block shape per GPU by hand (Sec. 3.4); here the shape
 * is data.  A zero field means "library default". */
typedef struct {
    int32_t dx, dy, dz;        /* spacing the entry applies to; 0 matches any value */
    int32_t adj_zchunk;        /* adjoint: tile-planes per warp unit, 3..16 (0: chosen per volume
                                  by the library's load-balance model) */
    int32_t adj_warps;         /* adjoint: warps per CTA, 1..4 (default 4, fewer if shared
                                  memory requires) */
    int32_t fwd_strip_tiles;   /* forward: tiles per warp strip, 4..29 (default 28 or 29,
                                  whichever keeps FP32 rows 16-byte aligned) */
    int32_t fwd_warps;         /* forward: warps per CTA, 1..8 (default 8, fewer if shared
                                  memory requires) */
} bsi_tile_config;

#define BSI_MAX_TILE_CONFIGS 256

/* Replaces the process-wide table (host memory, copied; n = 0 clears it).
 * Every later call plans with it: an instance takes the first entry whose
 * non-zero dx/dy/dz all match its spacing.  Because adj_zchunk changes the
 * adjoint workspace size, query the workspace after setting the table.
 * Returns BSI_ERR_BATCH for n outside 0..BSI_MAX_TILE_CONFIGS, BSI_ERR_SPACING
 * for a field out of range (the table is then left unchanged). */
bsi_status bsi_set_tile_configs(const bsi_tile_config* cfgs, int n);

/* The launch shape the library will use for spacing (dx, dy, dz), defaults
 * filled in except adj_zchunk and fwd_strip_tiles, which stay 0 when unset
 * because they depend on the volume; BSI_ERR_NULL if out is NULL,
 * BSI_ERR_SPACING for a bad spacing. */
bsi_status bsi_get_tile_config(int32_t dx, int32_t dy, int32_t dz, bsi_tile_config* out);

/* Static string naming a status code. */
const char* bsi_status_string(bsi_status s);

/* Message of the last CUDA error seen by this thread's calls ("" if none). */
const char* bsi_last_cuda_error(void);

/* Reads and clears the current device's kernel error word, synchronising
 * `stream` first (the one call that synchronises).  *flags receives the
 * word (0: no kernel recorded an error).  Returns BSI_ERR_DEVICE_STATUS if
 * it was non-zero, BSI_ERR_CUDA if the read failed. */
bsi_status bsi_check_device_status(bsi_stream_t stream, uint32_t* flags);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int bsi_version(void);

/* ------------------------------------------------------------------------
 * Non-integer, non-aligned spacing (Sec. 8 leaves control grids that are not
 * aligned to the voxel grid to future work, noting the weights must then be
 * computed on the fly).  Per axis (x, y, z) the spacing is num/den voxels and
 * the lattice is shifted by off/den voxels: voxel x has
 *   q = x den + off,  cell f = floor(q / num),  offset u = (q - f num) / num,
 * and Eq. 1 reads stored columns f .. f + 3 (the one-point border below, as
 * for integer spacing; den = 1, off = 0 is integer spacing).  Control point g
 * sits at voxel coordinate (g - 1) num/den - off/den.  Grid dims per axis:
 *   floor(((N - 1) den + off) / num) + 4.
 * Limits: 1 <= den <= BSI_MAX_RATIONAL_DEN, den <= num <= 64 den (spacing
 * 1..64), 0 <= off < num (BSI_ERR_SPACING); nx <= BSI_MAX_RATIONAL_NX (one
 * row of y/z-contracted columns lives in shared memory; BSI_ERR_DIMS).
 * ------------------------------------------------------------------------ */
#define BSI_MAX_RATIONAL_DEN 1024
#define BSI_MAX_RATIONAL_NX 16384

typedef struct {
    int64_t X, Y, Z;
    int32_t num[3], den[3], off[3];   /* (x, y, z) */
    int64_t nx, ny, nz;               /* stored grid, from bsi_geom_rational_init */
} bsi_geom_rational;

/* Fills g and its grid dims; BSI_ERR_DIMS / BSI_ERR_SPACING / BSI_ERR_NULL. */
bsi_status bsi_geom_rational_init(bsi_geom_rational* g, int64_t X, int64_t Y, int64_t Z, const int32_t num[3],
                                  const int32_t den[3], const int32_t off[3]);

/* Eq. 1 on such a grid, weights computed per voxel from the exact offset
 * (rounded once to FP32), FP32 output.
 *   phi   : device, FP32 [nz][ny][nx][3], read only
 *   field : device, FP32 [Z][Y][X][3], fully overwritten
 * BSI_ERR_GRID_MISMATCH if g's grid dims differ from the formula above; other
 * checks as bsi_field_forward.  One launch on `stream`. */
bsi_status bsi_field_forward_rational(const bsi_geom_rational* g, const float* phi, float* field,
                                      bsi_stream_t stream);

/* Workspace bytes bsi_field_adjoint_rational needs (partial sums: 6 KB per unit
 * of one z-cell part x one y-cell x a strip of up to 29 x-cells); 0 for an
 * invalid or empty geometry. */
size_t bsi_rational_adjoint_workspace_bytes(const bsi_geom_rational* g);

/* Transpose of bsi_field_forward_rational (the gradient of a loss with respect
 * to the grid, given grad_field = dL/dfield):
 *   grad_phi[g] = sum over voxels x of W(x, g) grad_field[x],
 * W(x, g) the product of the three axes' weights of bsi_field_forward_rational.
 * Deterministic (fixed summation order, no atomics): per-unit partial sums in
 * the workspace, then one sum per control point.
 *   grad_field : device, FP32 [Z][Y][X][3], read only
 *   grad_phi   : device, FP32 [nz][ny][nx][3], fully overwritten (zeros for an
 *                empty volume)
 *   workspace  : device, >= bsi_rational_adjoint_workspace_bytes(g) bytes,
 *                16-byte aligned; contents on entry ignored
 * Pointers 4-byte aligned (BSI_ERR_ALIGN); BSI_ERR_WORKSPACE for a missing or
 * short workspace; geometry checks as bsi_field_forward_rational.  Two
 * launches on `stream`. */
bsi_status bsi_field_adjoint_rational(const bsi_geom_rational* g, const float* grad_field, float* grad_phi,
                                      void* workspace, size_t workspace_bytes, bsi_stream_t stream);

/* The paper's own GPU formulations of Eq. 1, for its accuracy comparison
 * (Sec. 5.4) and as a measured contrast to the separable kernel:
 *   BSI_VARIANT_SEPARABLE  bsi_field_forward's strip kernel (FP32 output)
 *   BSI_VARIANT_TT         thread per tile (Sec. 3.2): the 64-term sum of Eq. 1
 *                          per channel, the cell's control points in registers
 *   BSI_VARIANT_TTLI       thread per tile with linear interpolations (Sec. 3.3,
 *                          App. B): 8 trilinear interpolations of 2x2x2
 *                          sub-cubes and one of their results, each lerp an FMA
 * phi and field as for bsi_field_forward (field FP32).  TT and TTLI take
 * spacings up to 32 (BSI_ERR_SPACING); an unknown variant is BSI_ERR_DTYPE.
 * TT and TTLI store each voxel from the thread that computes it, as the
 * paper's kernels do: they are not the fast path. */
typedef enum { BSI_VARIANT_SEPARABLE = 0, BSI_VARIANT_TT = 1, BSI_VARIANT_TTLI = 2 } bsi_variant;

bsi_status bsi_field_forward_variant(const bsi_geom* g, const float* phi, float* field, int32_t variant,
                                     bsi_stream_t stream);

/* Scalar BSI: Eq. 1 with one channel, for interpolating (zooming) an image
 * whose samples serve as the control points (Sec. 8 names image
 * interpolation as another use of the method).  The same kernels as
 * bsi_field_forward with a channel count of 1:
 *   out[z][y][x] = sum_{l,m,n} B_l(u) B_m(v) B_n(w) coeff[k+n][j+m][i+l]
 * with the geometry, border convention and spacing of bsi_field_forward.
 *   coeff : device, FP32 [nz][ny][nx], read only
 *   out   : device, [Z][Y][X] of out_dtype (BF16: round to nearest even of the
 *           FP32 result), fully overwritten
 * Same argument checks and error codes as bsi_field_forward. */
bsi_status bsi_scalar_forward(const bsi_geom* g, const float* coeff, void* out, bsi_dtype out_dtype,
                              bsi_stream_t stream);

/* ------------------------------------------------------------------------
 * BSI fused with the resampling of the floating image.
 *
 * In FFD registration the dense field of Eq. 1 exists to resample the
 * floating image (Sec. 6: NiftyReg interpolates the coarse control grid into
 * the fine deformation field, then warps the floating image with it); the
 * paper proposes merging such steps with BSI (Sec. 8).  These calls never
 * store the field: each voxel's displacement T(x) becomes the sample position
 *   p = x + T(x)   (voxel units; floating-image voxel i sits at coordinate i)
 * of the floating image F, read with the trilinear interpolant of F extended
 * by zeros outside it:
 *   F~(p) = sum over s, t, r in {0, 1} of
 *           (s ? a : 1 - a) (t ? b : 1 - b) (r ? c : 1 - c) F[k+r][j+t][i+s],
 *   i = floor(p_x), a = p_x - i (likewise j, b for y and k, c for z),
 *   F taken as 0 at indices outside [0, fX) x [0, fY) x [0, fZ).
 * F must be finite (a tap outside the image reads an in-range element with
 * weight 0).
 * ------------------------------------------------------------------------ */

/* Largest floating image, in elements (the kernels index it with 32-bit offsets). */
#define BSI_MAX_FLOATING_ELEMS 4294967295ull

/* warped[z][y][x] = F~(x + T_x, y + T_y, z + T_z).
 *   g        : reference volume (X, Y, Z) and spacing; phi [nz][ny][nx][3] on it
 *   floating : device, FP32 [fZ][fY][fX], fX, fY, fZ in 1..BSI_MAX_DIM and
 *              fX * fY * fZ <= BSI_MAX_FLOATING_ELEMS (else BSI_ERR_DIMS)
 *   warped   : device, FP32 [Z][Y][X], fully overwritten
 * Pointers 4-byte aligned (BSI_ERR_ALIGN), non-NULL (BSI_ERR_NULL; phi and
 * warped may be NULL for an empty volume).  One launch on `stream`. */
bsi_status bsi_resample_forward(const bsi_geom* g, const float* phi, const float* floating, int64_t fX,
                                int64_t fY, int64_t fZ, float* warped, bsi_stream_t stream);

/* Workspace bytes bsi_resample_backward needs: the voxel gradient G (12 B per
 * voxel, 256-byte aligned) followed by the adjoint's workspace (the bound of
 * bsi_adjoint_workspace_bytes).  0 for an empty volume. */
size_t bsi_resample_backward_workspace_bytes(const bsi_geom* g);

/* Gradient of a loss L(warped) with respect to phi, given grad_warped = dL/dwarped:
 *   G[z][y][x][c] = grad_warped[z][y][x] * dF~/dp_c (x + T(x))   (one-sided from
 *                   above at integer positions, where floor() puts them)
 *   grad_phi      = transpose of Eq. 1 applied to G (bsi_field_adjoint's sum)
 * Two stages: one fused launch (Eq. 1 + the interpolant's gradient) writes G
 * into the workspace, then the adjoint's two launches.
 *   grad_warped : device, FP32 [Z][Y][X]
 *   grad_phi    : device, FP32 [nz][ny][nx][3], fully overwritten
 *   workspace   : device, >= bsi_resample_backward_workspace_bytes(g) bytes,
 *                 16-byte aligned; contents on entry ignored
 * Same argument checks as bsi_resample_forward; BSI_ERR_WORKSPACE for a
 * missing or short workspace.  The gradient with respect to the floating
 * image is not computed. */
bsi_status bsi_resample_backward(const bsi_geom* g, const float* phi, const float* floating, int64_t fX,
                                 int64_t fY, int64_t fZ, const float* grad_warped, float* grad_phi,
                                 void* workspace, size_t workspace_bytes, bsi_stream_t stream);

/* Failure-detection self-test, no counterpart in the paper: enqueues one warp
 * that waits for a bulk copy that never comes -- it arms an mbarrier for 16
 * bytes and issues no copy -- with the same bounded wait the kernels use on
 * their copies (at most about 2 s).  When the wait gives up, the warp records
 * BSI_DEVICE_FLAG_TIMEOUT in the device status word, as a lost copy in a
 * kernel would, and returns: no fault, no trap, the context stays usable.
 * Read the result with bsi_check_device_status.  BSI_ERR_CUDA if the launch
 * fails. */
#define BSI_DEVICE_FLAG_TIMEOUT 128u
bsi_status bsi_selftest_lost_copy(bsi_stream_t stream);

/* Measurement utility, no counterpart in the paper: fills `bytes` bytes at
 * device address dst with the 32-bit pattern `value`, through the forward
 * kernel's store path (TMA bulk copies from shared memory, 16 KB each, from
 * every SM), so that its time gives the write-only HBM peak, the denominator
 * of the forward's store roofline.  dst and bytes must be multiples of 16
 * (BSI_ERR_ALIGN); dst NULL with bytes > 0 is BSI_ERR_NULL; bytes == 0 does
 * nothing.  Enqueued on `stream`, allocates nothing; BSI_ERR_CUDA if the launch
 * fails. */
bsi_status bsi_probe_fill(void* dst, size_t bytes, uint32_t value, bsi_stream_t stream);

/* Host-only diagnostic, no CUDA call: plans the launches of a batched call of
 * kind op (0 forward FP32, 1 forward BF16, 2 adjoint, 3 / 4 the resampling's
 * value / gradient launch, 5 / 6 the scalar forward FP32 / BF16, on each
 * instance's geometry) exactly as the entry
 * points do, and checks with the kernels' own index functions that every
 * global read and write lies inside its buffer and every staging copy fits
 * its shared-memory buffer.  With cover != 0 it also checks that the forward
 * writes each voxel exactly once and that the adjoint reduce reads only
 * partial sums its first kernel writes (host memory ~ volume size).
 * Returns the number of violations (0: all in range); the first one is
 * described in msg (may be NULL). */
int bsi_selfcheck_ranges(const bsi_instance* inst, int n, int op, int cover, char* msg, size_t msg_len);

#ifdef __cplusplus
}
#endif

#endif /* BSI_H */
