/*
 * gs.h - C ABI of the GB300 (sm_103a) tile-based Gaussian-splatting library.
 *
 * The library implements the rendering pipeline of 3D Gaussian Splatting as the
 * GEMM-GS paper describes it (Sec. 2.1: preprocessing, duplication, sorting,
 * blending) with the blending stage evaluated either per pixel on CUDA cores
 * (Alg. 1) or, following Sec. 3 (Eqs. 4-8, Alg. 2), as a tensor-core
 * contraction of per-splat coefficient rows v_g against intra-tile pixel
 * monomials v_p = [xb^2, yb^2, xb*yb, xb, yb, 1], followed by exp, the 1/255
 * skip, the 0.99 clamp and front-to-back compositing with early termination.
 *
 * Conventions for every entry point:
 *  - Pointers named in a call are DEVICE pointers unless the comment says HOST.
 *    The caller owns all memory; the library never allocates device memory and
 *    never frees what it is given.  Scratch space is passed in explicitly
 *    (gs_bin_sort) after a size query.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) unless its comment says it synchronises.
 *  - Arrays are dense, row-major, float32 unless stated.  Images are CHW:
 *    image[c * H * W + y * W + x].
 *  - Pixel (x, y) covers [x, x+1) x [y, y+1) and is evaluated at its centre
 *    (x + 0.5, y + 0.5).  Tiles are 16 x 16 pixels; tile t = ty * tiles_x + tx
 *    with tiles_x = ceil(W / 16), tiles_y = ceil(H / 16).
 *  - A return other than GS_OK leaves outputs unspecified.  Host-detectable
 *    errors (bad arguments, launch failures) are returned at once.  Faults the
 *    kernels detect (a device wait that exceeded its time limit) are recorded
 *    in a per-device error word that gs_sync_status() reads and clears.
 *  - Host threads may call the library at the same time, each on its own
 *    stream: launch shapes are computed once under a lock, and each persistent
 *    blend launch takes its own tile-queue slot (a pool of 1024).  Exceptions:
 *    gs_project_bin_small, gs_render_small and gs_bin_sort_noalloc calls must not overlap (one
 *    grid-barrier word, one scratch area), and the error word is shared, so
 *    gs_sync_status() may report another call's fault.
 *  - Calls that do not synchronise can be recorded in a CUDA graph.  The
 *    synchronising ones are gs_bin_sort, gs_bin_sort_noalloc and
 *    gs_bin_sort_views with a host count, gs_blend_autotune,
 *    gs_measure_peaks and gs_sync_status.  The first call of an entry point
 *    on a device sets kernel attributes and looks up device symbols: make it
 *    before any capture.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* gs_stream;

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,  /* null pointer, negative size, unknown option */
    GS_ERR_CUDA = 2,         /* a CUDA runtime call failed; see gs_last_error() */
    GS_ERR_CAPACITY = 3,     /* duplicated instances exceed the caller's capacity */
    GS_ERR_TIMEOUT = 4,      /* a device-side wait gave up after its time limit */
    GS_ERR_UNSUPPORTED = 5,  /* no sm_100-family GPU, or option not built */
    GS_ERR_WORKSPACE = 6     /* workspace smaller than the size query returned */
} gs_status;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).
 * p_cam = R p_world + t with world_to_cam = [R | t] row-major 3 x 4. */
typedef struct gs_camera {
    int32_t width, height;  /* pixels, >= 1 */
    float fx, fy, cx, cy;   /* focal lengths and principal point, pixels */
    float world_to_cam[12];
    float znear;            /* splats with camera z <= znear are culled (0.2 typical) */
    float lowpass;          /* added to both diagonal entries of the 2D covariance (0.3 typical) */
} gs_camera;

/* Blend arithmetic.  FP32 evaluates Eq. 3 per pixel on CUDA cores; the TC
 * variants evaluate Eq. 6 for a whole tile as a tcgen05 matrix product with
 * the given operand type and FP32 accumulation.  _SPLIT variants store v_g as
 * an unevaluated sum of 2 (fp16) or 3 (bf16) operand-type terms.  FP8_SPLIT
 * (a precision trial) uses e4m3 operands: every v_g row scaled by a power of
 * two and split into 5 terms, the pixel monomials into 2 exact terms.
 * PERSISTENT_FP32 is the TC variants' kernel (persistent tile queue, pixel
 * pairs, branch-free compositing, the same FP32 v_g rows of Eq. 6) with the
 * contraction v_g . v_p evaluated by FP32 FMAs on the CUDA cores instead of
 * tcgen05.mma: it isolates what the tensor cores contribute (forward only;
 * gs_blend_backward returns GS_ERR_UNSUPPORTED for it). */
typedef enum gs_variant {
    GS_BLEND_FP32 = 0,
    GS_BLEND_TC_FP16 = 1,
    GS_BLEND_TC_BF16 = 2,
    GS_BLEND_TC_FP16_SPLIT = 3,
    GS_BLEND_TC_BF16_SPLIT = 4,
    GS_BLEND_TC_FP8_SPLIT = 5,
    GS_BLEND_PERSISTENT_FP32 = 6
} gs_variant;

/* Options of the blend calls.  All-zero is valid: FP32 variant, defaults. */
typedef struct gs_blend_opts {
    int32_t variant;     /* gs_variant */
    int32_t chunk;       /* TC: splats per pipeline stage; 0 = default (32) */
    int32_t stages;      /* TC: depth of the shared-memory ring; 0 = default (2).
                            Built (chunk, stages): (32, 4), (32, 2), (16, 4), (16, 6) */
    int32_t ref_origin;  /* TC: reference pixel of each 16 x 8 half-tile (x0.., y0.. its
                            first pixel): 0 = its centre (x0 + 8, y0 + 4),
                            1 = the centre of its first pixel (x0 + 0.5, y0 + 0.5) */
    float bg[3];         /* background colour added as T_final * bg */
    int32_t bwd_stages;  /* TC backward: depth of its shared-memory ring, 0 = the variant's default
                            (6 for fp16 operands, 3 for bf16 and FP8, the deepest that keeps 3 blocks
                            per SM); built: 2, 3, 4, 6 (gs_blend_autotune_backward picks one) */
    int64_t timeout_ns;  /* limit of every device-side wait; 0 = 1 s */
    int32_t shard_count; /* tile sharding across ranks: the call blends only the tiles t
                            (global tile ids) with t % shard_count == shard_index and leaves
                            the other tiles' pixels untouched; the backward then adds only
                            those tiles' contributions, so the sum over shards is the full
                            gradient.  0 or 1 = all tiles */
    int32_t shard_index; /* 0 <= shard_index < max(1, shard_count) */
    const uint32_t* tile_order; /* NULL: tiles in id order.  Else a DEVICE array, a permutation of the
                                   call's global tile ids (e.g. from gs_tile_order): the kernels take
                                   the tile at position p of it in place of tile p, so persistent
                                   blocks start on the longest lists; with sharding, a shard takes the
                                   positions p with p % shard_count == shard_index.  It must have one
                                   entry per tile of the call; an entry >= the tile count is clamped
                                   (a wrong image, never an access outside the tile ranges) */
    uint64_t* issued_pairs;     /* NULL, or a DEVICE counter the tensor-core forward adds its issued
                                   Gaussian-pixel pairs to: 256 x the splats of every chunk it
                                   evaluates before a tile's exit (every pixel stopped), whether or
                                   not a pixel still needs them; the evaluated pairs of Eq. 1 are the
                                   sum of n_contrib.  The caller zeroes it */
    const float* splat_records; /* NULL, or a DEVICE table from gs_pack_splats over the call's items
                                   (the same mean2d, conic, opacity, rgb), 16-byte aligned: the
                                   tensor-core kernels then stage each chunk's splat records into
                                   shared memory with TMA gather copies (cp.async.bulk.tensor
                                   tile::gather4) issued chunks ahead, instead of loading the splat
                                   arrays thread by thread.  Same results bit for bit; ignored by the
                                   FP32 variant */
    int64_t splat_record_count; /* rows of splat_records (n_items of gs_pack_splats), 1 .. 2^31 - 1;
                                   a row beyond it reads as zeros, never outside the table */
} gs_blend_opts;

/* Library version (major * 100 + minor). */
int32_t gs_version(void);
/* Static text for a status code. */
const char* gs_status_string(gs_status status);
/* Text of the last failure on the calling host thread ("" if none). */
const char* gs_last_error(void);

/*
 * gs_project - preprocessing stage (Sec. 2.1 (a)): EWA projection of n 3D
 * Gaussians into one camera.
 *   means n x 3, scales n x 3 (linear standard deviations), quats n x 4
 *   (w, x, y, z; normalised inside), sh n x K x 3 with K = (sh_degree + 1)^2,
 *   sh_degree in 0..3.  `cam` is a HOST pointer.
 * Per Gaussian g (outputs n x 2, n x 3, n, n, n x 3, n):
 *   p = R mean + t; culled if p.z <= znear.  Sigma3 = (Rq S)(Rq S)^T;
 *   J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]];
 *   Sigma2 = (J R) Sigma3 (J R)^T + lowpass I = [[a, b], [b, c]];
 *   culled if det = ac - b^2 <= 0; conic = (c, -b, a) / det, evaluated in FP64
 *   when the FP32 det is below 1e-6;  mean2d = (fx x/z + cx, fy y/z + cy),
 *   culled if either coordinate exceeds 2^23 in magnitude;
 *   radius = min(ceil(3 sqrt(lambda_max(Sigma2))), 2^24);  depth = p.z;
 *   rgb = max(0, sum_k sh[g][k] Y_k(d) + 0.5), d = unit(mean - camera centre),
 *   Y_k the real spherical harmonics (sqrt(2) Re/Im of the complex ones with
 *   the Condon-Shortley phase, m = -l..l within degree l);
 *   tiles_touched = number of tiles of the rectangle
 *   [floor((mx - r)/16), floor((mx + r)/16)] x [same for y] clamped to the grid.
 * Culled Gaussians get radius 0 and tiles_touched 0.
 */
gs_status gs_project(int32_t n, const float* means, const float* scales, const float* quats,
                     const float* sh, int32_t sh_degree, const gs_camera* cam,
                     float* mean2d, float* conic, float* depth, int32_t* radius, float* rgb,
                     uint32_t* tiles_touched, gs_stream stream);

/*
 * gs_project_views - gs_project for n_views cameras in one launch (the batched
 * rendering of many views).  `cams` is a HOST array of n_views (1..32)
 * cameras; every output holds n_views blocks of n entries, view-major: view v,
 * Gaussian g at index v * n + g (mean2d [n_views][n][2], conic [n_views][n][3], ...).
 */
gs_status gs_project_views(int32_t n, const float* means, const float* scales, const float* quats,
                           const float* sh, int32_t sh_degree, const gs_camera* cams, int32_t n_views,
                           float* mean2d, float* conic, float* depth, int32_t* radius, float* rgb,
                           uint32_t* tiles_touched, gs_stream stream);

/*
 * gs_project_bin_small - gs_project and the per-tile lists of gs_bin_sort for
 * one camera in ONE cooperative launch, for small scenes (Sec. 2.1 (a)-(c);
 * the fusion is not in the paper).  For a few thousand to tens of thousands
 * of Gaussians the separate bin/sort stage is mostly launch latency; here the
 * blocks project every Gaussian, meet at a grid barrier, and each builds the
 * list of its tiles by gathering the splats that cover the tile and ordering
 * them by (depth bits, Gaussian index) in shared memory.  The gather scans all
 * n splats for every tile (O(tiles * n) work), so larger scenes belong to
 * gs_bin_sort.
 *   Inputs as gs_project (`cam` a HOST pointer); power_min NULL for the full
 *   rectangles, else one float per Gaussian (gs_alpha_power_min) for the
 *   opacity-aware lists of gs_bin_sort_views (the conics are the ones this
 *   call writes).  max_per_tile in 1..GS_SMALL_MAX_PER_TILE with
 *   tiles * max_per_tile < 2^32.
 *   Outputs: those of gs_project (mean2d 8-byte aligned); ids, tiles x
 *   max_per_tile: tile t's list at ids[t * max_per_tile ...]; tile_ranges
 *   (2 per tile) [t * max_per_tile, t * max_per_tile + count), so tile t's
 *   list is ids[tile_ranges[2t] .. tile_ranges[2t+1]) and equals gs_bin_sort's
 *   list of tile t, as the blend calls take it.
 * A tile with more than max_per_tile splats keeps an unspecified subset and
 * gs_sync_status() later returns GS_ERR_CAPACITY; a grid barrier that waited
 * longer than 1 s sets GS_ERR_TIMEOUT.  The grid barrier's counter is one
 * word in the library, so calls must not run concurrently.  Asynchronous.
 */
#define GS_SMALL_MAX_PER_TILE 16384
gs_status gs_project_bin_small(int32_t n, const float* means, const float* scales, const float* quats,
                               const float* sh, int32_t sh_degree, const gs_camera* cam, const float* power_min,
                               int32_t max_per_tile, float* mean2d, float* conic, float* depth, int32_t* radius,
                               float* rgb, uint32_t* tiles_touched, uint32_t* ids, uint32_t* tile_ranges,
                               gs_stream stream);

/*
 * gs_render_small - gs_project_bin_small and the blend forward of every tile
 * in the SAME cooperative launch: the fused project -> bin -> blend step for
 * small scenes, where the separate launches are mostly launch latency
 * (Sec. 2.1 (a)-(d) in one kernel; the fusion is not in the paper).  The
 * block that orders a tile's list blends that tile from the list it holds in
 * shared memory: Eq. 1 with Alg. 1's skip and stop rules, the exponents by
 * the contraction of Eq. 6 on the tensor cores, 32 splats per MMA, with the
 * operands and arithmetic of GS_BLEND_TC_FP16_SPLIT (centre reference
 * pixels).
 *   Inputs and outputs of gs_project_bin_small, plus opacity (n floats), bg
 *   (HOST, 3 floats) and the outputs of gs_blend_forward: image 3 x H x W,
 *   T_final H x W, n_contrib H x W (int32).  The images equal
 *   gs_blend_forward's (GS_BLEND_TC_FP16_SPLIT, ref_origin 0) on the same
 *   lists; gs_blend_backward takes T_final, n_contrib and the lists as they
 *   are.
 * Errors as gs_project_bin_small; a tensor-core wait that exceeded 1 s also
 * sets GS_ERR_TIMEOUT (the affected tiles are left unwritten).  Calls must
 * not run concurrently with each other or with gs_project_bin_small.
 * Asynchronous.
 */
gs_status gs_render_small(int32_t n, const float* means, const float* scales, const float* quats, const float* sh,
                          int32_t sh_degree, const gs_camera* cam, const float* power_min, int32_t max_per_tile,
                          const float* opacity, const float* bg, float* mean2d, float* conic, float* depth,
                          int32_t* radius, float* rgb, uint32_t* tiles_touched, uint32_t* ids, uint32_t* tile_ranges,
                          float* image, float* T_final, int32_t* n_contrib, gs_stream stream);

/*
 * gs_project_backward - gradient of gs_project_views (the preprocessing stage
 * of Sec. 2.1 (a); the paper has no backward pass), summed over the views.
 *   Inputs: the forward's inputs (means, scales, quats, sh, sh_degree, cams,
 *   n_views; `cams` a HOST array), its radius output (n_views x n, view-major:
 *   view v, Gaussian g at v * n + g; radius 0 = culled, no gradient) and the
 *   loss gradient of its outputs in the same layout: dmean2d n_views x n x 2
 *   (8-byte aligned), dconic n_views x n x 3 (the entries A, B, C of the conic
 *   [[A, B], [B, C]]), drgb n_views x n x 3 (e.g. gs_blend_backward's outputs).
 *   Outputs (overwritten): dmeans n x 3, dscales n x 3, dquats n x 4 (of the
 *   quaternions as given, before normalisation), dsh n x K x 3.
 * Chain rule through conic = Sigma2^-1, Sigma2 = (J R) Rq S S^T Rq^T (J R)^T
 * + lowpass I with J at p = R mean + t, mean2d, the normalisation q / |q| and
 * the SH colour rgb = max(0, sum_k sh_k Y_k(d) + 0.5) (a channel clamped at 0
 * passes no gradient; the view direction d depends on the mean).  FP32, one
 * thread per Gaussian; the 2x2 inverse's step in FP64 where the forward used
 * FP64 (determinant below 1e-6).  Asynchronous.
 */
gs_status gs_project_backward(int32_t n, const float* means, const float* scales, const float* quats,
                              const float* sh, int32_t sh_degree, const gs_camera* cams, int32_t n_views,
                              const int32_t* radius, const float* dmean2d, const float* dconic, const float* drgb,
                              float* dmeans, float* dscales, float* dquats, float* dsh, gs_stream stream);

/* Bytes of scratch gs_bin_sort needs for n Gaussians, `capacity` instances and
 * a width x height image.  `bytes` is a HOST pointer.  For gs_bin_sort_views
 * pass n = n_views * n_per_view (the size does not depend on the image). */
gs_status gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t width, int32_t height,
                                     size_t* bytes);

/*
 * gs_bin_sort - duplication and sorting stages (Sec. 2.1 (b), (c)).
 * Every Gaussian with radius > 0 is duplicated once per tile of its rectangle
 * (the rule of gs_project) with key (tile << 32) | float_bits(depth); the
 * instances are sorted by key, equal keys in Gaussian-index order (the order a
 * stable sort of the Gaussian-major, row-major-tile duplication gives).
 *   keys_sorted[capacity] (u64; may be NULL: the blend calls read only the
 *   ids and ranges, and without keys the last kernel writes 8 bytes less
 *   per instance), ids_sorted[capacity] (u32 Gaussian index),
 *   tile_ranges[2 * num_tiles] (u32 [start, end) per tile, empty = [0, 0)).
 *   workspace: device scratch of at least gs_bin_sort_workspace_size() bytes,
 *   256-byte aligned; its contents on entry do not matter.
 *   n_instances: HOST pointer, receives the number of instances I.
 * This call synchronises `stream` once (to read I).  If I > capacity it
 * returns GS_ERR_CAPACITY with *n_instances = I and writes no sorted output.
 * Requires capacity < 2^32.
 */
gs_status gs_bin_sort(int32_t n, const float* mean2d, const int32_t* radius, const float* depth,
                      int32_t width, int32_t height, int64_t capacity,
                      void* workspace, size_t workspace_bytes,
                      uint64_t* keys_sorted, uint32_t* ids_sorted, uint32_t* tile_ranges,
                      int64_t* n_instances, gs_stream stream);

/*
 * gs_bin_sort_views - gs_bin_sort over the items of n_views views at once.
 * Items are (view, Gaussian) pairs, item = v * n_per_view + g, laid out as
 * gs_project_views writes them; widths/heights are HOST arrays.  View v owns
 * the global tiles [T_v, T_v + tiles_x(v) * tiles_y(v)) with T_v the tile
 * count of the views before it; keys carry the global tile id and ids_sorted
 * the item index; tile_ranges has 2 * (total tiles) entries.
 * Two modes:
 *  - n_instances != NULL (HOST): as gs_bin_sort, synchronises once;
 *  - n_instances == NULL, n_instances_dev != NULL (device int64): never
 *    synchronises, so it can be captured in a CUDA graph.  Grids are sized by
 *    `capacity`; the instance count is written to *n_instances_dev; if it
 *    exceeds capacity the lists are truncated and gs_sync_status() later
 *    returns GS_ERR_CAPACITY.
 * Opacity-aware lists (the tighter tile intersection; not in the paper): with
 * conic (the items' conics, 3 floats each, as gs_project writes them) and
 * power_min (one float per Gaussian, from gs_alpha_power_min) a splat keeps a
 * tile of its rectangle only if its exponent can reach power_min somewhere in
 * the tile's box of pixel-centre offsets, i.e. if that box meets the region
 * q(d) = A dx^2 + 2 B dx dy + C dy^2 <= -2 power_min; each rectangle row keeps
 * one run of tiles, found in closed form from the region's extent within the
 * row (an ellipse, or for a nearly singular or indefinite conic, as needle-
 * shaped splats give, a band around its null line).  Dropped splats would
 * fail the 1/255 test at every pixel of the tile, so images and T_final are
 * those of the full lists (n_contrib counts list positions and shrinks).  The
 * rule is FP32 with one rounding per operation in a fixed order, so the lists
 * are reproducible bit for bit; against the exact (FP64) decision they differ
 * only on pairs whose box lies within rounding of the threshold.  A or C <= 0
 * keeps the whole rectangle; power_min >= 0 keeps no tile.  Both NULL: the
 * full rectangles.
 */
gs_status gs_bin_sort_views(int32_t n_views, int32_t n_per_view, const float* mean2d, const int32_t* radius,
                            const float* depth, const float* conic, const float* power_min,
                            const int32_t* widths, const int32_t* heights, int64_t capacity,
                            void* workspace, size_t workspace_bytes, uint64_t* keys_sorted, uint32_t* ids_sorted,
                            uint32_t* tile_ranges, int64_t* n_instances, int64_t* n_instances_dev,
                            gs_stream stream);

/*
 * gs_tile_order - the global tile ids of n_views views (widths/heights HOST
 * arrays, as gs_bin_sort_views) ordered longest list first, from a sorted
 * list's tile_ranges, into tile_order (one uint32 per tile) for
 * gs_blend_opts.tile_order (not in the paper: a scheduling aid).  Persistent
 * blend blocks take tiles from a queue; taking the longest lists first keeps
 * the last blocks from finishing long after the others.  Buckets of a
 * quarter octave of list length, longest bucket first; the order within a
 * bucket is unspecified (the images do not depend on it).  One block, one
 * launch; asynchronous.
 */
gs_status gs_tile_order(int32_t n_views, const int32_t* widths, const int32_t* heights, const uint32_t* tile_ranges,
                        uint32_t* tile_order, gs_stream stream);

/* power_min[g] = ln(1 / (255 opacity[g])) - 2e-3 (+inf when opacity < 1.0f/255.0f)
 * for n Gaussians: the exponent a splat must reach somewhere in a tile for
 * alpha >= 1/255 there, lowered by a margin above the exponent error of the
 * FP32 and split tensor-core blends.  Device pointers; asynchronous. */
gs_status gs_alpha_power_min(int32_t n, const float* opacity, float* power_min, gs_stream stream);

/*
 * gs_pack_splats - the splat parameters the blends read, packed per item into
 * one 64-byte record (not in the paper: the data layout of the staged,
 * pipelined splat loads of Sec. 3.4 on this GPU), for gs_blend_opts.splat_records.
 * Items are view-major as in the *_views calls: item v * n_per_view + g.
 *   mean2d n_items x 2, conic n_items x 3, rgb n_items x 3 (may be NULL: zero
 *   colour), opacity n_per_view (indexed by g): DEVICE inputs.
 *   records: DEVICE output, n_items x 16 floats, 16-byte aligned:
 *   [mx, my, A, B, C, log2 o, min(log2 o, log2 0.99), 1/o, r, g, b, g (bits), 0, 0, 0, 0]
 *   (log2 0 = -inf, 1/0 = 0).  One launch; asynchronous.
 */
gs_status gs_pack_splats(int32_t n_items, int32_t n_per_view, const float* mean2d, const float* conic,
                         const float* opacity, const float* rgb, float* records, gs_stream stream);

/*
 * gs_bin_sort_noalloc - gs_bin_sort for callers that cannot allocate device
 * memory (the paper has no counterpart: it is a deployment convenience).
 * Some callers get only their input and output buffers: code inside a host
 * framework whose allocator owns the device, plugins, or processes with a
 * memory budget fixed in advance.  This entry point takes no workspace; its
 * scratch is one array of gs_bin_sort_noalloc_max_bytes() bytes (64 MiB)
 * compiled into the library, which every device that loads the library holds
 * until the process exits.  Arguments and results are those of gs_bin_sort.
 *  - Returns GS_ERR_WORKSPACE, writing nothing, if gs_bin_sort_workspace_size
 *    (n, capacity, width, height) exceeds that size.
 *  - It calls no allocation routine.  The first call on a device looks up
 *    the array's device address (once per device, that device current); make
 *    that first call before any stream capture.
 *  - Rejects with GS_ERR_INVALID_ARG, before any CUDA call, what gs_bin_sort
 *    rejects: a side outside 1..2^20, an image of 2^31 tiles or more, null
 *    pointers.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 *    The array's previous contents never matter (everything read is written
 *    first within the call).
 *  - The array's device address is kept for the life of the process: a
 *    cudaDeviceReset between calls is not supported (the same holds for the
 *    library's error word).
 */
size_t gs_bin_sort_noalloc_max_bytes(void);
gs_status gs_bin_sort_noalloc(int32_t n, const float* mean2d, const int32_t* radius, const float* depth,
                              int32_t width, int32_t height, int64_t capacity, uint64_t* keys_sorted,
                              uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_instances,
                              gs_stream stream);

/*
 * gs_blend_forward - blending stage (Eq. 1; Alg. 1 for GS_BLEND_FP32, Alg. 2
 * with Eqs. 6-8 for the TC variants).  For every pixel, over its tile's list
 * in order: power = -1/2 (A dx^2 + C dy^2) - B dx dy (dx = mx - x, dy = my - y);
 * alpha = min(0.99, o exp(min(power, 0))); the splat is skipped if
 * alpha < 1/255; with T' = T (1 - alpha), compositing stops before the splat
 * if T' < 1e-4; otherwise C += rgb alpha T and T = T'.
 *   mean2d n x 2, conic n x 3 (A, B, C), opacity n, rgb n x 3: per Gaussian.
 *   image 3 x H x W = C + T bg;  T_final H x W;  n_contrib H x W (int32) =
 *   1 + list position of the last splat added, 0 if none.
 * `opts` is a HOST pointer (NULL = all defaults).
 */
gs_status gs_blend_forward(int32_t width, int32_t height, const uint32_t* tile_ranges,
                           const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                           const float* opacity, const float* rgb, const gs_blend_opts* opts,
                           float* image, float* T_final, int32_t* n_contrib, gs_stream stream);

/*
 * gs_blend_backward - gradient of the blended image with respect to each
 * Gaussian's mean2d, conic, opacity and rgb, given dL_dimage (3 x H x W) and
 * the forward call's T_final and n_contrib.  Each pixel walks its list back to
 * front from n_contrib - 1, recovering T_i = T_{i+1} / (1 - alpha_i) and the
 * colour behind splat i, S_i (S = bg after the last splat,
 * S_{i-1} = alpha_i c_i + (1 - alpha_i) S_i):
 *   dL/dc_i = alpha_i T_i g,  dL/dalpha_i = T_i (c_i - S_i) . g,
 *   dalpha/do = e^p and dalpha/dp = alpha (both 0 where the 0.99 clamp holds),
 *   dp/dmx = -(A dx + B dy), dp/dmy = -(B dx + C dy),
 *   dp/dA = -dx^2/2, dp/dB = -dx dy, dp/dC = -dy^2/2.
 * alpha is recomputed with the arithmetic of the forward call's variant, so
 * the backward pass skips and stops exactly where the forward did:
 *  - GS_BLEND_FP32: the FP32 quadratic of Eq. 3 (Alg. 1), one block per tile;
 *  - every tensor-core variant: the forward's own Eq. 6 contraction on the
 *    tensor cores (the same v_g rows and operand terms, FP32 accumulate); the
 *    per-splat sums over a tile's pixels (dL/dpower times the monomials, and
 *    the colour weights) are a second tensor-core contraction with fp16
 *    operands (dL/dpower as fp16 hi + lo, the weight alpha T as one fp16).
 * Pass the same opts->variant as the forward call that produced T_final and
 * n_contrib.  Gradients are ADDED (atomically) to dmean2d n x 2, dconic n x 3,
 * dopacity n, drgb n x 3: zero them first.
 */
gs_status gs_blend_backward(int32_t width, int32_t height, const uint32_t* tile_ranges,
                            const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                            const float* opacity, const float* rgb, const gs_blend_opts* opts,
                            const float* T_final, const int32_t* n_contrib, const float* dL_dimage,
                            float* dmean2d, float* dconic, float* dopacity, float* drgb,
                            gs_stream stream);

/*
 * gs_blend_forward_views / gs_blend_backward_views - the blend of n_views
 * views in one launch; for the tensor-core variants one persistent launch
 * walks a single queue over the tiles of all views.  Inputs as produced by
 * gs_project_views + gs_bin_sort_views (mean2d, conic, rgb per item; opacity
 * per Gaussian, n_per_view entries).  Images are packed view after view:
 * image holds 3 x H_v x W_v floats per view (CHW) starting at 3 * P_v, and
 * T_final / n_contrib H_v x W_v entries starting at P_v, where P_v is the
 * pixel count of the views before v; dL_dimage is laid out like image.
 * Gradients: dmean2d / dconic / drgb per item, dopacity per Gaussian (summed
 * over views).
 */
gs_status gs_blend_forward_views(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                 int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                 const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                 const gs_blend_opts* opts, float* image, float* T_final, int32_t* n_contrib,
                                 gs_stream stream);
gs_status gs_blend_backward_views(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                  int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                  const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                  const gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                                  const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity,
                                  float* drgb, gs_stream stream);

/*
 * gs_blend_autotune - pick the pipeline shape of a tensor-core blend by
 * measurement: runs gs_blend_forward_views once per built (chunk, stages)
 * pair (one warm-up, then `reps` timed runs with CUDA events on `stream`) and
 * writes the fastest pair into opts->chunk / opts->stages (opts is a HOST
 * pointer; its variant must be a TC variant).  image / T_final / n_contrib
 * are overwritten.  Synchronises the stream.  *best_ms (HOST, may be NULL)
 * receives the mean time of the chosen pair.
 */
gs_status gs_blend_autotune(int32_t n_views, const int32_t* widths, const int32_t* heights, int32_t n_per_view,
                            const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                            const float* conic, const float* opacity, const float* rgb, gs_blend_opts* opts,
                            float* image, float* T_final, int32_t* n_contrib, int32_t reps, float* best_ms,
                            gs_stream stream);

/*
 * gs_blend_autotune_backward - the same for the tensor-core backward pass:
 * runs gs_blend_backward_views with each built ring depth (bwd_stages 2, 3,
 * 4, 6), `reps` timed calls each, and sets opts->bwd_stages to the fastest
 * (not in the paper: its batch-size study, Sec. 4.4, picks the mini-batch
 * shape by measurement).  Arguments as gs_blend_backward_views; the gradient
 * buffers are accumulated into many times, so their contents afterwards are
 * unspecified: zero them before the real call.  Synchronises `stream`.
 */
gs_status gs_blend_autotune_backward(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                     int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                     const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                     gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                                     const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity,
                                     float* drgb, int32_t reps, float* best_ms, gs_stream stream);

/*
 * gs_tile_power - the exponent matrix M_power = M_g . M_p of Eq. 8 exactly as a
 * TC variant's blend computes it, for inspection and testing.  For each of the
 * n_tiles tiles in `tiles` (device int32), every list position j < max_len and
 * tile pixel p = 16 * row + col: out[(i * max_len + j) * 256 + p] =
 * log2(e) * power + log2(opacity), the base-2 exponent the blend feeds to exp2.
 * Positions past a tile's list are left untouched.  opts->variant must be a
 * TC variant.
 */
gs_status gs_tile_power(int32_t width, int32_t height, const uint32_t* tile_ranges,
                        const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                        const float* opacity, const gs_blend_opts* opts, const int32_t* tiles,
                        int32_t n_tiles, int32_t max_len, float* out, gs_stream stream);

/* Number of kernels this library has launched in the calling process (all
 * devices, all host threads), for accounting of GPU work. */
int64_t gs_launch_count(void);

/*
 * gs_set_kernel_events - timing of one kernel inside a library call (for
 * profiling; the paper has no counterpart).  While set, every call that
 * launches `kernel` records the CUDA event `start` (a cudaEvent_t) on its
 * stream just before that launch and `end` just after it (during a stream
 * capture as external event records, so that every replay of the graph
 * records them): the elapsed time between them is the kernel's duration.
 * An error of the record (e.g. an event of another device) fails the call
 * with GS_ERR_CUDA.  kernel: GS_KERNEL_DUPLICATE,
 * the coarse duplication of gs_bin_sort / gs_bin_sort_views /
 * gs_bin_sort_noalloc.  start and end both NULL clear the setting; both must
 * be events of the device the calls run on.  Process-wide: calls that run
 * concurrently record into the same events.
 */
#define GS_KERNEL_DUPLICATE 1
gs_status gs_set_kernel_events(int32_t kernel, void* start, void* end);

/* Synchronise `stream`, then return and clear the device error word of the
 * current device: GS_ERR_TIMEOUT if a kernel's bounded wait gave up since the
 * last call, else GS_OK (or GS_ERR_CUDA if synchronising failed). */
gs_status gs_sync_status(gs_stream stream);

/* Self-test of the bounded device wait used by the tensor-core pipeline: one
 * CTA waits on an mbarrier that nothing ever arrives on, gives up after
 * timeout_ns (capped at 1 s) and records GS_ERR_TIMEOUT in the error word,
 * which gs_sync_status() then returns. */
gs_status gs_selftest_bounded_wait(int64_t timeout_ns, gs_stream stream);

/* Measured peaks of the units that bound the blend kernels (the paper has no
 * counterpart; it is how rooflines here get their denominators).  Rates are
 * whole-GPU operations per second at the clock the GPU ran at meanwhile. */
typedef struct {
    double ex2_per_s;  /* MUFU ex2.approx.f32 results per second */
    double rcp_per_s;  /* MUFU rcp.approx.f32 results per second */
    double fma_per_s;  /* FP32 fused multiply-adds per second (2 FLOPs each) */
    double sm_mhz;     /* mean SM clock during the three measurements (clock64 / globaltimer) */
    int32_t sms;       /* streaming multiprocessors */
} gs_peaks;

/* Run the microbenchmarks on the current device: each fills every thread slot
 * of every SM with 8 independent dependent chains of one operation and takes
 * the best of 3 timed launches (about 20 ms in all).  `out` is a HOST pointer.
 * Synchronises `stream`; uses a small scratch array compiled into the library
 * (calls that overlap on the GPU race on it, harmlessly for the timing). */
gs_status gs_measure_peaks(gs_peaks* out, gs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
