/*
 * vdi.h -- C ABI of the GB300 library for distributed Volumetric Depth Image
 * (VDI) generation and compositing.
 *
 * Method: Gupta et al., "Parallel Compositing of Volumetric Depth Images for
 * Interactive Visualization of Distributed Volumes at High Frame Rates".
 * Each processing element (PE) owns one box of the volume's cells.  Phase 1
 * raycasts every PE's box from a shared camera into a compact sub-VDI (sec. 4,
 * sec. 5.1); phase 2 composites the K sub-VDIs of each pixel into one regular
 * VDI of at most N_S supersegments (sec. 5.2, Eq. 2, Algorithm S1).  On one
 * GPU all K sub-VDIs live in device memory; the paper's all-to-all exchange
 * is the composite kernel's per-pixel gather.
 *
 * Conventions shared by every entry point:
 *   - All array arguments are DEVICE pointers unless marked "host".  The
 *     caller allocates and frees every buffer; the library allocates no
 *     device memory in any entry point and frees nothing it did not create.
 *   - Calls are asynchronous on `stream` (0 = the legacy default stream) and
 *     do not synchronise the host, except where a flag asks for it.
 *   - Errors are returned as vdi_status; no C++ exception crosses the ABI.
 *     Argument errors are detected on the host before any launch.  Errors a
 *     kernel detects (an output buffer too small) are written to a status
 *     word inside the caller's workspace; vdi_workspace_status() reads it.
 *     vdi_last_error() returns a message for the last failing call on the
 *     calling host thread.
 *   - Depth is distance from the eye along the unit ray direction, in voxel
 *     units.  The volume's nodes sit at integer coordinates 0..dims-1; cell
 *     (i,j,k) spans [i,i+1] x [j,j+1] x [k,k+1].
 *   - A supersegment ("record") is {front f, back b, premultiplied R,G,B,
 *     opacity A}.  FP32 records are stored as two arrays, float4 rgba[] and
 *     float2 fb[] (24 bytes); FP16 records as one array of 16-byte structs
 *     {float f; float b; half r, g, b, tau;}: premultiplied colour in IEEE
 *     binary16, the opacity as its base-2 optical depth tau = -log2(1 - A)
 *     in binary16 (A = 1 - 2^-tau; tau = +inf for A = 1), depth in FP32.
 *     tau keeps the opacity's relative precision at every value: binary16 A
 *     itself would round every A above 1 - 2^-12 to an opaque 1 and move the
 *     extinction -log2(1 - A) / (b - f) of the compositing mixture by up to
 *     its whole value.  Kernels accumulate in FP32 either way.
 */
#ifndef VDI_H
#define VDI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vdi_stream; /* same type as cudaStream_t */

typedef enum {
    VDI_OK = 0,
    VDI_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is invalid */
    VDI_ERR_CAPACITY = 2,    /* an output buffer holds fewer records than needed */
    VDI_ERR_WORKSPACE = 3,   /* the workspace is smaller than the query said */
    VDI_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    VDI_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    VDI_ERR_MODEL = 6,       /* a learned-gamma model is missing or malformed */
    VDI_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} vdi_status;

typedef enum { VDI_PREC_F32 = 0, VDI_PREC_F16 = 1 } vdi_precision;
typedef enum { VDI_VOL_F32 = 0, VDI_VOL_U16 = 1 } vdi_voltype;

/* Maximum number of PEs in one call. */
#define VDI_MAX_PE 64

/* gamma modes of vdi_generate / vdi_choose_gamma */
#define VDI_GAMMA_SEARCH (-1.0f) /* per-ray bisection search (sec. 2.4) */
#define VDI_GAMMA_GIVEN (-2.0f)  /* per-ray gamma read from vdi_compact.gamma */
#define VDI_GAMMA_CHOSEN (-3.0f) /* vdi_generate only: counts and gamma already written by vdi_choose_gamma */

/* One PE's owned cells: [lo, hi) per axis, x, y, z. */
typedef struct {
    int32_t lo[3], hi[3];
} vdi_box;

/* Pinhole camera (host struct).  Pixel (i, j), j = 0 the top row, gets the ray
 * through its centre: d = normalize(fwd + x right + y up'), x = (2(i+1/2)/W - 1)
 * tan(fovy/2) W/H, y = (1 - 2(j+1/2)/H) tan(fovy/2), fwd = normalize(center -
 * eye), right = normalize(fwd x up), up' = right x fwd. */
typedef struct {
    double eye[3], center[3], up[3];
    double fovy_deg;
    int32_t width, height;
} vdi_camera;

/* Sampling parameters (host struct).  Samples lie on a grid shared by all PEs:
 * sample k of a ray covers [t_in + k step, t_in + (k+1) step] with midpoint
 * t_in + (k + 1/2) step, t_in the ray's entry into the whole volume's box, for
 * every k whose midpoint lies before the exit.  A sample belongs to the PE
 * whose box holds the cell floor(midpoint) (clamped to the volume's cells).
 * The transfer function's opacity is given per ref_len voxels and corrected to
 * the step (sec. 2.4, "length-adjusted opacity"). */
typedef struct {
    float step;           /* sample spacing in voxels, > 0 */
    float ref_len;        /* length the table's opacity refers to, > 0 */
    int32_t bisect_iters; /* bisection steps of the gamma search, 1..24 (16) */
    int32_t schedule;     /* 0: automatic; see vdi_composite */
    int32_t flags;        /* VDI_FLAG_* */
} vdi_params;

#define VDI_FLAG_SYNC_CAPACITY 1 /* vdi_generate: read totals back and return VDI_ERR_CAPACITY before emitting */
#define VDI_FLAG_CENSUS 2        /* vdi_choose_gamma / vdi_generate / vdi_composite: count the work done (vdi_workspace_counters) */
#define VDI_FLAG_LEARNED_SINGLE_PASS 4 /* vdi_choose_gamma_learned: no bracketed refinement (see there) */

/* A sampling brick: one PE's cells in the library's cell-packed layout, built
 * by vdi_brick_build().  Opaque to the caller apart from its size. */
typedef struct {
    const float* cells; /* device, vdi_brick_bytes() bytes */
    vdi_box owned;      /* the PE's cells */
    int32_t dims[3];    /* nodes of the whole volume per axis */
    float value_scale;  /* stored value * value_scale = v in [0,1] */
} vdi_brick;

/* Compact sub-VDI of one PE (sec. 4, Fig. 2c).  For pixel p = j*W + i the
 * records are [offsets[p], offsets[p] + counts[p]).  vdi_generate writes
 * offsets as the exclusive prefix sum of counts (offsets[W*H] = total);
 * vdi_composite reads only offsets[p] and counts[p], so any start layout
 * (several PEs sharing one record pool, say) is accepted there. */
typedef struct {
    uint32_t* counts;  /* [W*H] */
    uint64_t* offsets; /* [W*H + 1] */
    void* rgba;        /* F32: float4[capacity]; F16: 16-byte records[capacity] */
    float* fb;         /* F32: float2[capacity]; F16: unused (NULL) */
    float* gamma;      /* [W*H] per-ray gamma (output of generation; input in VDI_GAMMA_GIVEN mode) */
    uint64_t capacity; /* records the record arrays hold */
    int32_t prec;      /* vdi_precision */
} vdi_compact;

/* Regular VDI (sec. 4, Fig. 2a): N_S slots per pixel, pixel-major, front to
 * back, unused slots zero; counts[p] slots used.  Record (p, j) is at index
 * p * n_s + j. */
typedef struct {
    uint32_t* counts; /* [W*H] */
    void* rgba;       /* F32: float4[W*H*n_s]; F16: 16-byte records[W*H*n_s] */
    float* fb;        /* F32: float2[W*H*n_s]; F16: unused (NULL) */
    float* gamma;     /* [W*H] gamma chosen by the compositing search, or NULL */
    int32_t n_s;
    int32_t prec; /* vdi_precision */
} vdi_regular;

/* ------------------------------------------------------------------------ */
/* Version, errors                                                          */
/* ------------------------------------------------------------------------ */
int32_t vdi_version(void);
const char* vdi_status_string(vdi_status s);
/* Copies the message of the last failing call on this host thread into buf
 * (at most n bytes, NUL-terminated) and returns that call's status. */
vdi_status vdi_last_error(char* buf, size_t n);
/* Synchronises `stream`, reads the device status word in `workspace` and
 * returns it (VDI_OK if no kernel reported an error since the call that last
 * cleared it; every entry point taking a workspace clears it first). */
vdi_status vdi_workspace_status(const void* workspace, vdi_stream stream);
/* Synchronises `stream` and copies the work counters of the last call made
 * with VDI_FLAG_CENSUS on this workspace into counters[8] (host):
 *   [0] samples evaluated (trilinear + classification), summed over marches,
 *   [1] state-machine steps (samples x gamma candidates evaluated),
 *   [2] marches over a ray's samples, [3] (PE, ray) pairs with samples,
 *   [4] pairs that needed the bisection search, [5] of those, pairs whose
 *   non-transparent samples did not fit the sample cache, [6] marches over
 *   cached samples, [7] marches re-sampling the volume for the search.
 * After vdi_composite with the flag the counters are instead:
 *   [0] pixels, [1] pixels that needed the search, [2] sweeps over a
 *   pixel's pieces (search marches plus the emitting sweep), [3] pieces
 *   visited over those sweeps, [4] state-machine steps (pieces x gamma
 *   candidates), [5] input records, [6] bisection levels answered by the
 *   decision intervals of earlier marches, [7] unused.
 * The census runs a separately compiled variant of the kernel; without the
 * flag nothing is counted. */
vdi_status vdi_workspace_counters(const void* workspace, uint64_t counters[8], vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Decomposition and bricks (sec. 3: blocks as close to equal as the data    */
/* dimensions permit)                                                        */
/* ------------------------------------------------------------------------ */
/* Near-equal split of the cells of a dims[0] x dims[1] x dims[2] node volume
 * into grid[0]*grid[1]*grid[2] boxes (x fastest).  Host only.  boxes_out
 * (host) receives the boxes.  Cell runs along an axis differ by at most one. */
vdi_status vdi_split_boxes(const int32_t dims[3], const int32_t grid[3], vdi_box* boxes_out);

/* Bytes of the sampling brick of box `owned` (32 bytes per cell, including a
 * one-cell border). */
size_t vdi_brick_bytes(const vdi_box* owned);

/* Builds the sampling bricks of k PEs from the whole volume `volume` (device,
 * node values x fastest, type `type`: float32 v in [0,1] or uint16 v = u/65535).
 * cells_out[e] (host array of k device pointers) receives vdi_brick_bytes(&boxes[e])
 * bytes each; bricks_out (host, k entries) is filled in.  One launch. */
vdi_status vdi_brick_build(const void* volume, vdi_voltype type, const int32_t dims[3], int32_t k,
                           const vdi_box* boxes, float* const* cells_out, vdi_brick* bricks_out, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Phase 1: sub-VDI generation (sec. 4, sec. 5.1, Eq. 1)                     */
/* ------------------------------------------------------------------------ */
/* Workspace bytes for vdi_generate / vdi_choose_gamma with k PEs of w x h on
 * the current device: a status header, a work counter, the prefix sum's
 * partial sums (8 bytes per 4096 pixels per PE), a sample cache (1024
 * entries of 8 bytes per resident thread: 152 SMs x 12 CTAs x 64 threads,
 * about 0.96 GB, on a GB300) that lets the gamma search run over each ray's
 * cached non-transparent samples instead of re-sampling the volume, and each
 * (PE, ray)'s recorded span (8 bytes per PE and pixel, plus 256): the samples
 * from its first to its last non-transparent one, which emission marches
 * instead of all of the ray's samples in the PE's box.  Any workspace of at
 * least 512 bytes plus 8 k ceil(w h / 4096) rounded up to a multiple of 256
 * is accepted, with the same results: without room for the cache the search
 * re-marches the volume, without room for the spans emission marches every
 * sample (slower). */
size_t vdi_generate_workspace(int32_t k, int32_t w, int32_t h);

/* Chooses gamma and the resulting supersegment count for every (PE, ray)
 * without emitting records: out[e].gamma and out[e].counts are written.
 * gamma >= 0: that value for every ray; VDI_GAMMA_SEARCH: per-ray bisection
 * (gamma = 0 if it yields at most n_s, else bisection of [0, 2] for
 * params->bisect_iters steps, stopping early at exactly n_s; the upper end is
 * returned); VDI_GAMMA_GIVEN: out[e].gamma is read, and rays whose count at
 * that gamma exceeds n_s fall back to the search.  counts are the number of
 * records emission at that gamma produces with the budget n_s. */
vdi_status vdi_choose_gamma(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                            int32_t n_s, float gamma, vdi_compact* out, const vdi_params* params, void* workspace,
                            size_t ws_bytes, vdi_stream stream);

/* Generates the k compact sub-VDIs: vdi_choose_gamma, the exclusive prefix sum
 * of the counts into offsets (sec. 4), and emission of the records.
 * tf_lut: device float[256*4], straight RGB and opacity per ref_len.
 * gamma as in vdi_choose_gamma, or VDI_GAMMA_CHOSEN to skip choosing: out[e].counts
 * and out[e].gamma then hold the result of an earlier vdi_choose_gamma call
 * with the same bricks, camera, n_s and params (only the prefix sum and the
 * emission run).  Emission marches the spans the last choice on this
 * workspace recorded when that choice had the same bricks, table, camera and
 * sampling parameters (compared as values: pointers, boxes, camera, step),
 * and every sample otherwise.  A caller that rewrites the bricks' or the
 * table's contents in place between vdi_choose_gamma and this call must
 * choose again, or pass another workspace.
 * Records of a list are in depth order, at most n_s per list for box-shaped
 * domains.  If a PE's total exceeds out[e].capacity, no record past the
 * capacity is written and VDI_ERR_CAPACITY is reported through the workspace
 * status (or returned, with offsets valid, under VDI_FLAG_SYNC_CAPACITY); in
 * the first case the counts of the lists the capacity cuts are reduced to the
 * records written, so the sub-VDI remains valid input for vdi_composite. */
vdi_status vdi_generate(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                        int32_t n_s, float gamma, vdi_compact* out, const vdi_params* params, void* workspace,
                        size_t ws_bytes, vdi_stream stream);
/* Sub-VDIs in the regular layout instead (sec. 4: the layout earlier VDI
 * generation used; Table 1 compares its generation time and memory with the
 * compact layout's):
 * out[e] (k descriptors, n_s slots per pixel, one precision) receives PE e's
 * counts, gamma and records at p * n_s with a zero tail.  No prefix sum and
 * no capacity question: every pixel owns n_s slots.  gamma as for
 * vdi_generate, except VDI_GAMMA_CHOSEN.  Workspace as vdi_generate. */
vdi_status vdi_generate_regular(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                                int32_t n_s, float gamma, vdi_regular* out, const vdi_params* params,
                                void* workspace, size_t ws_bytes, vdi_stream stream);

/* Non-convex decompositions (sec. 5.3): ownership given per block of cells
 * instead of by boxes.  owner[(bz * nb[1] + by) * nb[0] + bx] (device, one
 * byte per block, x fastest) is the PE owning the block's cells; a value >= k
 * means no PE.  block: edge of a block in cells, a power of two 1..1024;
 * nb[a] = ceil((dims[a] - 1) / block). */
typedef struct {
    const uint8_t* owner;
    int32_t block;
    int32_t nb[3];
} vdi_ownership;
/* vdi_generate under an ownership map: bricks[e].owned must contain every
 * cell PE e owns (its blocks' bounding box, say); PE e keeps the samples whose
 * cell it owns.  Where a ray leaves PE e's domain and comes back, the open
 * supersegment ends there, and the next non-transparent sample opens a new
 * one even when n_s have been opened: a list may then hold more than n_s
 * records (one per domain run at gamma = 2, the flat-DVR limit of sec. 5.3),
 * and the search returns gamma = 2 with that count when no gamma meets n_s.
 * gamma >= 0, VDI_GAMMA_SEARCH or VDI_GAMMA_GIVEN; other arguments, outputs
 * and errors as vdi_generate. */
vdi_status vdi_generate_owned(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                              int32_t n_s, float gamma, const vdi_ownership* own, vdi_compact* out,
                              const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Batched generation: many generation requests (their own volumes, cameras, */
/* image sizes, K, N_S and gamma modes) in one persistent launch.  No        */
/* counterpart in the paper, where every PE generates its own sub-VDI for    */
/* one frame (sec. 5.1); the per-(PE, ray) work is that of vdi_generate.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    const vdi_brick* bricks; /* host array of k bricks (device cells inside); one volume per request */
    int32_t k;               /* PEs of the request, 1..VDI_MAX_PE */
    const float* tf_lut;     /* device float[256*4] */
    vdi_camera cam;          /* the request's camera and image size */
    int32_t n_s;             /* supersegments per list */
    float gamma;             /* >= 0 fixed, VDI_GAMMA_SEARCH or VDI_GAMMA_GIVEN */
    vdi_compact* out;        /* host array of k sub-VDI descriptors (device arrays inside), one precision */
} vdi_gen_request;

/* Bytes of the table of n requests (host query). */
size_t vdi_gen_batch_table_bytes(const vdi_gen_request* reqs, int32_t n);
/* Checks the requests as vdi_generate checks its arguments and packs them,
 * with params (step, ref_len, bisect_iters; flags and schedule unused), into
 * host_table (host, vdi_gen_batch_table_bytes bytes).  The caller copies the
 * table to device memory (dev_table); both are passed to
 * vdi_generate_batched.  The table holds the requests' device pointers: a
 * new table is needed when buffers move. */
vdi_status vdi_gen_batch_table_pack(const vdi_gen_request* reqs, int32_t n, const vdi_params* params,
                                    void* host_table, size_t bytes);
/* Workspace bytes for a packed table: 512 bytes of status and counter, the
 * prefix sums' partial sums (8 bytes per 4096 pixels per PE) and the sample
 * cache of vdi_generate_workspace (the search re-marches the volume when the
 * workspace has no room for it; same result). */
size_t vdi_generate_batched_workspace(const void* host_table);
/* Generates every request's k compact sub-VDIs: one persistent launch in
 * which CTAs take (request, PE, 16 x 4-pixel tile) items from an atomic
 * counter in the workspace (reset by this call with a stream-ordered memset)
 * and choose gamma and the count of every ray of the item; one batched
 * exclusive prefix sum of every (request, PE) list; one launch emitting the
 * records.  The outputs equal those of one vdi_generate call per request,
 * bit for bit.  Capacity overflows and emission errors are reported through
 * the workspace status (vdi_workspace_status), as vdi_generate without
 * VDI_FLAG_SYNC_CAPACITY; nothing is read back, so the memset and the
 * launches can be captured in a CUDA graph and replayed. */
vdi_status vdi_generate_batched(const void* dev_table, const void* host_table, void* workspace, size_t ws_bytes,
                                vdi_stream stream);

/* Generation for callers that cannot allocate device memory (an in-situ
 * simulation that reserves its whole device budget at start-up, a plugin with
 * no access to its host application's allocator).  The paper has no
 * counterpart; this is vdi_generate with its workspace replaced by a static
 * device array inside the library (512 B + 512 KiB, held on every GPU that
 * loads the library until the process exits).  Nothing is allocated or freed.
 * The array has no room for the sample cache, so the gamma search re-marches
 * the volume (same result as vdi_generate, slower).
 *   - Limit: k * ceil(W*H / 4096) <= 65536 (e.g. 64 PEs at 2048 x 2048);
 *     larger requests return VDI_ERR_INVALID_ARG without touching the GPU.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     in the CUDA context current at that call, so another context on the
 *     same device, or one re-created after cudaDeviceReset, gets its own
 *     copy.  The first call in a context loads the library's device code;
 *     make that first call before any stream capture begins.
 *   - The call synchronises `stream`: it reads the K totals back and returns
 *     VDI_ERR_CAPACITY before emitting (VDI_FLAG_SYNC_CAPACITY is implied),
 *     and after emission it reads the status word the kernels write into the
 *     array and returns it (an inconsistent VDI_GAMMA_CHOSEN count, say, is
 *     VDI_ERR_CUDA), since the caller cannot read that word.
 *   - Every call uses the same array and leaves the previous call's contents
 *     in it (the status header is cleared by each call); calls that overlap
 *     on the GPU (several streams or host threads at once) race on it.
 * Arguments and outputs are those of vdi_generate. */
vdi_status vdi_generate_static_scratch(const vdi_brick* bricks, int32_t k, const float* tf_lut,
                                       const vdi_camera* cam, int32_t n_s, float gamma, vdi_compact* out,
                                       const vdi_params* params, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Phase 2: compositing (sec. 5.2, Eq. 2, Algorithm S1)                      */
/* ------------------------------------------------------------------------ */
/* Composites the k compact sub-VDIs (pe[e], all w x h) into the regular VDI
 * `out` (out->n_s slots per pixel).  Per pixel: the records of all lists with
 * b > f are cut at every front and back depth; an interval covered by one
 * record whole keeps that record, a part of one record gets the opacity of
 * Eq. 2, an interval covered by several records their emission-absorption
 * mixture, an uncovered interval between records is a transparent sample.
 * The pieces are re-segmented with Eq. 1 and a per-pixel gamma search, and
 * at most n_s supersegments are written front to back with a zero tail.
 * params->schedule (all give the same result, bit for bit):
 *   0 automatic (VDI_SCHED_LANE for k <= 8, else VDI_SCHED_STAGED);
 *   VDI_SCHED_STAGED (4, the pooled schedule): a warp builds the pieces of
 *     32 pixels, one pixel at a time with all its lanes (coalesced loads of
 *     the K lists, a stable merge of their bounds, an exact prefix scan of
 *     the records' terms), writes each pixel's pieces as one run of a pool in
 *     the workspace and lists the pixel; a second launch runs the search and
 *     the emission of every listed pixel, one lane each, lanes taking new
 *     pixels as they finish; pixels with more than 1024 records or lists out
 *     of depth order are composited by a direct sweep in a third launch.  The
 *     image is processed in chunks of pixels whose pieces fit the pool;
 *   VDI_SCHED_LANE (5, k <= 8; larger k take VDI_SCHED_STAGED): a warp copies
 *     the records of 32 consecutive pixels into shared memory with coalesced
 *     loads and each lane sweeps its pixel's lists there once: a pixel whose
 *     count at gamma = 0 is within n_s is emitted at once, a pixel that needs
 *     the search writes its pieces to the pool and is listed; the list is
 *     sorted by piece count (three small launches) and searched as in the
 *     pooled schedule; pixels whose records exceed the warp's 480-record slab,
 *     or whose pieces do not fit the pool, take a direct sweep;
 *   1, 2, 3 (direct): each thread sweeps its pixel's K lists on every march;
 *     1: list heads in registers (k <= 8), two bisection levels per march;
 *     2: heads in shared memory under a winner tree, two levels per march;
 *     3: as 2 with three levels per march.
 * Workspace: vdi_composite_workspace bytes hold the larger of the lane
 * schedule's needs (two lists of 16 bytes per pixel, 8 KB of sort scratch and
 * a pool of 16 pieces of 24 bytes per pixel) and the pooled schedule's (a
 * chunk of up to 131072 pixels with room for 2048 pieces each).  An automatic
 * schedule falls back to a direct one when the workspace is smaller; the
 * direct schedules need 256 bytes.  Colours must be non-negative
 * (premultiplied, at most A); a record's extinction -log2(1 - A) / (b - f) is
 * clamped at 2^56 per unit depth. */
#define VDI_SCHED_STAGED 4
#define VDI_SCHED_LANE 5
size_t vdi_composite_workspace(int32_t k, int32_t w, int32_t h, int32_t n_s);
vdi_status vdi_composite(const vdi_compact* pe, int32_t k, int32_t w, int32_t h, vdi_regular* out,
                         const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Batched compositing: many requests (image sizes, K, N_S) in the same     */
/* persistent launches.  No counterpart in the paper (which composites one  */
/* VDI per MPI rank); the per-pixel work is that of vdi_composite.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const vdi_compact* pe; /* host array of k sub-VDI descriptors (device pointers inside) */
    int32_t k, w, h;
    vdi_regular out;   /* the request's output (device pointers inside) */
    int32_t schedule;  /* as params->schedule of vdi_composite; 0 automatic */
} vdi_request;

/* Bytes of the request table of n requests (host query). */
size_t vdi_batch_table_bytes(const vdi_request* reqs, int32_t n);
/* Packs the requests into host_table (host, vdi_batch_table_bytes bytes).  The
 * caller copies it to device memory (dev_table) before the launch; both are
 * passed to vdi_composite_batched.  All requests must share one input
 * precision. */
vdi_status vdi_batch_table_pack(const vdi_request* reqs, int32_t n, void* host_table, size_t bytes);
/* Workspace bytes for a packed table (host_table from vdi_batch_table_pack). */
size_t vdi_composite_batched_workspace(const void* host_table);
/* Composites every request of the table with the pooled schedule run over all
 * of them at once: a persistent build launch in which warps take (request,
 * 32-pixel batch) items from an atomic counter in the workspace and write
 * every request's pieces to one pool, a search launch whose lanes take the
 * listed pixels of every request, and a launch of the direct sweep for the
 * pixels the stage cannot hold and the requests with a direct schedule (1-3,
 * run as 2).  The (request, pixel) list is processed in chunks of at most
 * 2^22 pixels whose pieces fit the pool.  Counters are reset with
 * stream-ordered memsets; the memsets and the launches may be captured into a
 * CUDA graph and replayed; the outputs equal those of one vdi_composite call
 * per request, bit for bit. */
vdi_status vdi_composite_batched(const void* dev_table, const void* host_table, const vdi_params* params,
                                 void* workspace, size_t ws_bytes, vdi_stream stream);
/* Autotuner: for each request whose schedule is 0, times the applicable
 * schedules (1 when k <= 8, 2, 3, and VDI_SCHED_STAGED when the workspace
 * holds vdi_composite_workspace(k, m, 1, n_s) bytes, m = min(w h, 2^20)) on
 * the first m of the request's pixels with CUDA events and stores the
 * fastest in
 * reqs[i].schedule.  Results are cached per (K bucket, N_S bucket, input
 * precision) for the life of the process, so later requests of the same
 * shape reuse them.  Synchronises the stream; overwrites the requests'
 * outputs. */
vdi_status vdi_composite_autotune(vdi_request* reqs, int32_t n, const vdi_params* params, void* workspace,
                                  size_t ws_bytes, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Learned gamma.  No counterpart in the paper, which searches gamma per ray */
/* (sec. 2.4); the search stays as the fallback and as the source of the     */
/* training labels.  A small MLP predicts log2 gamma per (PE, 16 x 16 tile)  */
/* from features of the tile's rays.                                          */
/* ------------------------------------------------------------------------ */
#define VDI_NFEAT 40       /* features per (PE, tile) */
#define VDI_GAMMA_TILE 16  /* tile edge in pixels; tiles are row-major, ceil(W/16) per row */

/* Model: one caller-allocated device buffer of vdi_model_bytes() bytes holding
 * the FP32 master parameters (vdi_model_nparams() = 6849: W1[64][40], b1[64],
 * W2[64][64], b2[64], w3[64], b3), their BF16 copy used by inference, the Adam
 * moments, the Adam step count and the init seed. */
size_t vdi_model_bytes(void);
int32_t vdi_model_nparams(void);
/* He-uniform weights from a counter-based generator (seed), zero biases and moments. */
vdi_status vdi_model_init(void* model, uint64_t seed, vdi_stream stream);
/* Checkpoint: synchronous copy of the whole buffer to / from a file
 * ("VDIMLP01" header, version, parameter count, size).  Training resumed from
 * a checkpoint continues bit for bit. */
vdi_status vdi_model_save(const void* model, const char* path, vdi_stream stream);
vdi_status vdi_model_load(void* model, const char* path, vdi_stream stream);

/* Features of every (PE, tile) from the owned samples of the tile's rays at
 * even pixel offsets (8 x 8 rays): [0..31] histogram of the opacity of
 * non-transparent samples (bins of 1/64, the last open), normalised; [32],
 * [33] mean and standard deviation of the first non-transparent sample's
 * depth from the PE's first sample, over the volume diagonal; [34], [35] the
 * same for the back of the last one; [36] log1p(mean non-transparent samples
 * per ray with samples) / 8; [37] n_s / 64; [38] fraction of those rays with a
 * non-transparent sample; [39] mean |P_k - P_prev| of consecutive
 * non-transparent samples.  feats: device float[k][tiles][40]; valid: device
 * uint8[k][tiles], 0 for tiles whose rays own no sample (features all 0). */
vdi_status vdi_tile_features(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                             int32_t n_s, const vdi_params* params, float* feats, uint8_t* valid, vdi_stream stream);
/* Training labels from a searched generation (searched[e].counts, .gamma):
 * per tile, the lower median over rays with a supersegment of
 * log2(max(gamma, 2^-20)).  labels: float[k][tiles]; valid: uint8[k][tiles]. */
vdi_status vdi_tile_labels(const vdi_compact* searched, int32_t k, int32_t w, int32_t h, float* labels,
                           uint8_t* valid, vdi_stream stream);
/* Inference on the tensor cores: log2_gamma[r] = MLP(feats[r]) - offset, n rows. */
vdi_status vdi_mlp_infer(const void* model, const float* feats, int32_t n, float offset, float* log2_gamma,
                         vdi_stream stream);
/* Training (FP32 arithmetic, BF16-rounded weights).  Loss: mean squared error
 * of the prediction over the rows with valid != 0.  vdi_mlp_grad writes the
 * gradient (device float[6849]) and the loss (device float); vdi_mlp_train_step
 * also applies one Adam step (beta 0.9, 0.999, eps 1e-8, learning rate lr).
 * Deterministic (per-block partial sums in the workspace, fixed-order reduction). */
size_t vdi_mlp_train_workspace(int32_t n);
vdi_status vdi_mlp_grad(const void* model, const float* feats, const float* labels, const uint8_t* valid, int32_t n,
                        float* grad, float* loss, void* workspace, size_t ws_bytes, vdi_stream stream);
vdi_status vdi_mlp_train_step(void* model, const float* feats, const float* labels, const uint8_t* valid, int32_t n,
                              float lr, float* loss, void* workspace, size_t ws_bytes, vdi_stream stream);
/* Learned gamma for generation: tile features, inference, then per ray one
 * march over the volume that counts at the tile's prediction gp =
 * 2^(output - offset) and caches the ray's non-transparent samples.  The
 * prediction then brackets a short search over the cached samples: log2 gamma
 * in [log2 gp - 4, log2 gp] when gp is feasible (count <= n_s), else
 * [log2 gp, log2 gp + 4] when its top is; six bisection levels (three cached
 * marches) give the smallest feasible gamma found.  Rays with no feasible
 * gamma in the bracket, or too many non-transparent samples for the cache, run
 * the full bisection search; rays with at most n_s non-transparent samples
 * take gamma = 0 as in the search.  Writes out[e].gamma and out[e].counts like
 * vdi_choose_gamma; follow with vdi_generate(..., VDI_GAMMA_CHOSEN, ...) to
 * emit.  The supersegment counts differ from the full search's only through
 * the bracket's resolution (a factor 2^(1/16) in gamma).
 * With VDI_FLAG_LEARNED_SINGLE_PASS in params->flags the prediction is used
 * as it is: one march per ray counts at gp, a ray within the budget keeps gp
 * and its count, and only rays over the budget run the full bisection search
 * (VDI_GAMMA_GIVEN with the predictions). */
size_t vdi_learned_workspace(int32_t k, int32_t w, int32_t h);
vdi_status vdi_choose_gamma_learned(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                                    int32_t n_s, const void* model, float offset, vdi_compact* out,
                                    const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Rendering a regular VDI (sec. 2.3: exact from its viewpoint of           */
/* generation by associativity of "over"; from other viewpoints the paper  */
/* judges VDIs against DVR but does not restate the renderer)               */
/* ------------------------------------------------------------------------ */
/* `vdi` is w x h pixels of camera `gen`.  With `view` NULL or equal to
 * `gen`: flattens each pixel's supersegments front to back into rgba_out
 * (device float4[w*h], premultiplied).  With another `view`: renders the
 * VDI as a view-dependent volume into rgba_out (device float4[view->width *
 * view->height], premultiplied; gen->width == w and gen->height == h):
 * pixel (i, j)'s frustum column (the points whose projection through gen's
 * eye falls in the pixel's square) holds its supersegments, each filling the
 * points at distance f..b from gen's eye with opacity 1 - (1 - A)^(l /
 * (b - f)) over a path of length l (the length correction of Eq. 2) and
 * straight colour P / A; each view ray is cut at column faces and shells
 * and composited front to back.  Stream-ordered, no allocation. */
vdi_status vdi_render_view(const vdi_regular* vdi, int32_t w, int32_t h, const vdi_camera* gen,
                           const vdi_camera* view, float* rgba_out, vdi_stream stream);

/* ------------------------------------------------------------------------ */
/* Frame pipeline (sec. 7: sub-VDI generation of the next VDI overlaps the   */
/* final gather of the previous one).  On one GPU the final gather is the    */
/* device-to-host copy of the composited regular VDI; the pipeline also     */
/* overlaps the host-to-device copy of the next time step's volume.          */
/* ------------------------------------------------------------------------ */
/* Per frame: volume upload (copy-in stream), brick build, generation and
 * compositing (compute stream), regular-VDI download (copy-out stream).  The
 * volume and the regular VDI are double-buffered in device memory, so frame
 * f + 1's upload and generation run while frame f's download is in flight.
 * Results equal those of vdi_brick_build, vdi_generate and vdi_composite
 * called in order on one stream, bit for bit. */
typedef struct vdi_pipeline vdi_pipeline; /* opaque, host-side */

typedef struct {
    int32_t dims[3];      /* nodes of the volume per axis */
    int32_t type;         /* vdi_voltype of the uploaded volumes */
    int32_t k;            /* PEs, 1..VDI_MAX_PE */
    vdi_box boxes[VDI_MAX_PE]; /* the PEs' cells (first k used) */
    int32_t width, height;
    int32_t n_s;          /* supersegments per list, sub-VDIs and output */
    int32_t prec;         /* vdi_precision of the sub-VDIs and the output */
    float gamma;          /* VDI_GAMMA_SEARCH or a fixed gamma >= 0 */
    uint64_t capacity;    /* records per PE sub-VDI; 0: width * height * n_s
                             (always enough for box-shaped domains) */
    vdi_params params;    /* schedule 0: autotuned on the first frame */
} vdi_pipeline_desc;

/* Device bytes of the arena a pipeline with this description needs (two
 * volumes, the k bricks, the k compact sub-VDIs, two regular VDIs, the
 * generation and compositing workspaces, two 8-byte status snapshots).  0 for
 * an invalid description. */
size_t vdi_pipeline_arena_bytes(const vdi_pipeline_desc* desc);
/* Creates a pipeline on the current device.  arena: caller-allocated device
 * memory of vdi_pipeline_arena_bytes(desc) bytes, 256-byte aligned, owned by
 * the caller and used until vdi_pipeline_destroy.  tf_lut (device
 * float[256*4]) is copied into the arena after a device-wide synchronisation
 * (so the table and the arena may come from any stream); creation is not
 * stream-ordered and must not be captured in a graph.  The pipeline creates three
 * non-blocking streams, its events and a small page-locked status mirror;
 * *out receives the handle.  One host thread at a time may use a pipeline. */
vdi_status vdi_pipeline_create(const vdi_pipeline_desc* desc, void* arena, size_t arena_bytes, const float* tf_lut,
                               vdi_pipeline** out);
/* Submits one frame and returns without waiting for it, once the frame two
 * submissions back has completed (at most two frames in flight; that
 * frame's status is then held for vdi_pipeline_wait).
 *   volume: HOST pointer to the frame's volume (dims, type), or NULL to keep
 *     the previous frame's volume and bricks (a camera-only frame; invalid on
 *     the first frame).  Read until the frame's upload has run: keep it
 *     unchanged until vdi_pipeline_wait(ticket) returns.
 *   cam: the frame's camera (width x height of the description), copied.
 *   dst: HOST buffers receiving the regular VDI (counts[W*H], rgba and, for
 *     FP32, fb of W*H*n_s records; gamma[W*H] if non-NULL); n_s and prec must
 *     be the description's.  Written asynchronously; valid after
 *     vdi_pipeline_wait(ticket).
 *   ticket: receives the frame's number (0, 1, 2, ...).
 * Host buffers should be page-locked: pageable copies do not overlap. */
vdi_status vdi_pipeline_submit(vdi_pipeline* pl, const void* volume, const vdi_camera* cam, const vdi_regular* dst,
                               uint64_t* ticket);
/* Waits for frame `ticket` (and all frames before it) and returns its status:
 * the status words the generation and compositing kernels left for that
 * frame (VDI_ERR_CAPACITY when a sub-VDI overflowed its capacity), or the
 * error of a CUDA call.  A ticket not yet submitted is VDI_ERR_INVALID_ARG.
 * For a ticket older than the last two, the first error of any earlier
 * frame is returned (VDI_OK if none). */
vdi_status vdi_pipeline_wait(vdi_pipeline* pl, uint64_t ticket);
/* The pipeline's copy-in, compute and copy-out streams (streams[3], host),
 * for ordering other work or timing events against the pipeline. */
vdi_status vdi_pipeline_streams(const vdi_pipeline* pl, vdi_stream streams[3]);
/* Waits for every submitted frame and releases the streams, events and
 * status mirror.  The arena is the caller's to free afterwards. */
vdi_status vdi_pipeline_destroy(vdi_pipeline* pl);

#ifdef __cplusplus
}
#endif
#endif /* VDI_H */
