/*
 * hasf.h -- C ABI of a GB300 (sm_103a) implementation of the homotopic
 * alternating sequential filter (HASF) of Mahmoudi & Akil, "Real Time
 * Topological Image Smoothing On Shared Memory Parallel Machines"
 * (arXiv:1603.09337).
 *
 * What the filter computes (Sec. 2 of the paper).  For a binary image X, a set
 * of kept points C within X and a set of forbidden points D outside X,
 *     HASF_n^{C,D} = HF_n^D o HC_n^C o ... o HF_1^D o HC_1^C,
 * where HC_r^C (homotopic cutting, eq. (i)) and HF_r^D (homotopic filling,
 * eq. (ii)) are a homotopic opening and closing by the Euclidean disc B_r,
 * built from exact squared Euclidean distance maps (Sec. 4.1), ball erosion and
 * dilation, and constrained thinning H / thickening *H that remove or add
 * simple points only (Sec. 2, Sec. 4.2).  Topology is preserved: the numbers of
 * n-components of X and nbar-components of its complement never change.
 *
 * Fixed readings where the paper is silent (every result is a pure function of
 * X, C, D, rmax and connectivity):
 *  - everything outside the image box is background and never changes;
 *  - H and *H take points by increasing priority level (squared distance,
 *    computed once on the operator's input), and within a level repeat rounds
 *    until nothing changes; a round visits the four 2x2 subfields
 *    (x mod 2, y mod 2) = (0,0), (1,0), (0,1), (1,1) in that order;
 *  - in eq. (ii), W = eps_r(Z) cup X (the printed eps_n(Y) names an undefined Y).
 *
 * Memory.  All image pointers are DEVICE pointers unless an entry point says
 * otherwise.  Images are row-major uint8, one byte per pixel, rows `pitch`
 * bytes apart; a non-zero byte is an object pixel.  Outputs are written as
 * 0/1 bytes.  The caller owns every image buffer; the library reads and writes
 * them only during the call's device work and keeps no reference afterwards
 * (for hasf_submit: until hasf_poll reports the job done).  The library owns
 * its scratch memory, which is taken from the context's byte budget.
 *
 * Errors.  Every entry point returns a hasf_status and never aborts the
 * process.  Argument errors are reported before any device work is issued.
 * Device-side outcomes (an iteration cap or a wait deadline: HASF_ETIMEOUT;
 * a run to stability that reached its cap: HASF_EUNSTABLE) are reported by
 * the next synchronising call (hasf_status_of / hasf_poll / the host-buffer
 * entry points); a CUDA runtime error is HASF_ECUDA.
 *
 * Streams.  `stream` arguments are cudaStream_t values passed as void*
 * (NULL = the legacy default stream).  Calls on one context must be issued to
 * one stream at a time, or be ordered by the caller: they share the context's
 * scratch memory.
 */
#ifndef HASF_H_
#define HASF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HASF_OK = 0,
    HASF_EINVAL = 1,      /* bad argument                                   */
    HASF_ENOMEM = 2,      /* a device or host allocation failed             */
    HASF_EBUDGET = 3,     /* the job can never fit the context's budget     */
    HASF_EPENDING = 4,    /* a submitted job is not finished yet            */
    HASF_ETIMEOUT = 5,    /* a device iteration cap or wait deadline hit    */
    HASF_ECUDA = 6,       /* a CUDA runtime call failed                     */
    HASF_ENOTFOUND = 7,   /* unknown ticket                                 */
    HASF_ECANCELLED = 8,  /* the job was cancelled before it ran            */
    HASF_EUNSTABLE = 9    /* run to stability: still changing at the cap    */
} hasf_status;

/* rmax for the filter run to stability with the largest cap (see hasf_image). */
#define HASF_RMAX_STABLE (-64)

/* One image to smooth.  in/out/C/D share `pitch`.  out may equal in.
 * C == NULL means C is empty; C is used as C cap X (Sec. 2 requires C within X).
 * D == NULL means D is empty; D is used as D minus X (Sec. 2 requires D in the
 * complement of X).  width, height in [1, 65536]; pitch >= width;
 * rmax in [1, 64] is the order n of the filter; connectivity is 8 for
 * (8,4) adjacency (8-connected object, 4-connected background) or 4 for (4,8).
 * rmax in [-64, -1] runs the filter to stability, the reading taken of the
 * unbounded radius ("r = infinity") of Table 1: steps r = 1, 2, ... (each
 * HC_r^C then HF_r^D) until one leaves the image unchanged, at most -rmax
 * steps.  out receives the image after the last step run; if step -rmax still
 * changed it, the job's status is HASF_EUNSTABLE (reported like
 * HASF_ETIMEOUT; a timeout takes precedence).  Such images run on the
 * register kernel when they are at most 512 x 512 and -rmax <= 31, else on the
 * generic kernels, with one more h * ceil(w / 32)-word plane of scratch. */
typedef struct hasf_image {
    const uint8_t *in;
    uint8_t *out;
    const uint8_t *C;
    const uint8_t *D;
    int32_t width;
    int32_t height;
    int32_t pitch;
    int32_t rmax;
    int32_t connectivity;
    int32_t reserved;     /* must be 0 */
} hasf_image;

typedef struct hasf_ctx hasf_ctx;

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * device scratch the context may hold (0 = 20 GiB).  *ctx receives the handle.
 * Errors: HASF_EINVAL (ctx NULL, bad device), HASF_ENOMEM, HASF_ECUDA. */
int hasf_create(hasf_ctx **ctx, int device, size_t mem_budget_bytes);

/* Wait for the context's device work, then free everything it owns.
 * Jobs submitted and not yet finished are cancelled first. */
int hasf_destroy(hasf_ctx *ctx);

/* Smooth one image, asynchronously on `stream`: HASF_rmax^{C,D}(in) -> out.
 * Errors: HASF_EINVAL (see hasf_image), HASF_EBUDGET, HASF_ENOMEM,
 * HASF_ECUDA.  A device-side HASF_ETIMEOUT is reported by hasf_status_of. */
int hasf_smooth(hasf_ctx *ctx, const hasf_image *img, void *stream);

/* Smooth n independent images in one persistent launch on `stream`.  `imgs`
 * is a HOST array of n descriptors (each holding device pointers); it may be
 * reused as soon as the call returns.  Images may differ in size, rmax,
 * connectivity and constraints.  The result of each image is the same as
 * hasf_smooth on it alone.  Buffers of different images must not overlap.
 * Errors as hasf_smooth; n = 0 is a no-op. */
int hasf_smooth_batch(hasf_ctx *ctx, const hasf_image *imgs, int n, void *stream);

/* Synchronise `stream` and report the device status of the context's last
 * launches on it: HASF_OK, HASF_ETIMEOUT or HASF_EUNSTABLE (and clear it), or
 * HASF_ECUDA. */
int hasf_status_of(hasf_ctx *ctx, void *stream);

/* Host-buffer form: every pointer in `imgs` is a HOST pointer (ordinary or
 * pinned memory).  By default (HASF_OPT_HOST_MAPPED 2) the register kernel
 * (images of at most 512 x 512, rmax <= 31), which reads each input byte once
 * and writes each output byte once, reads and writes the callers' buffers
 * itself, across the host link, with no staging copies: any buffer when the
 * device can access all host memory through the host's page tables (as on
 * GB300 with NVLink-C2C: cudaDevAttrPageableMemoryAccess), else the buffers
 * that are page-locked and mapped into the device's address space
 * (cudaHostAlloc, or cudaHostRegister with the mapped flag).  Mapped buffers
 * of larger images (and, under HASF_OPT_HOST_MAPPED 1, all mapped buffers)
 * move with one launch of the library's copy kernel per direction.  Other
 * buffers are staged through the context's pinned buffer with one copy per
 * buffer.  Synchronous: the results are in the callers' buffers on
 * return.  The buffers must not be freed or changed during the call.
 * Errors as hasf_smooth_batch, plus HASF_ETIMEOUT. */
int hasf_smooth_host(hasf_ctx *ctx, const hasf_image *imgs, int n);

/* Serving.  Submit one job (device pointers, which must stay valid until
 * hasf_poll reports it done).  Jobs are admitted as device slots and budget
 * free up and run batched with the other jobs in flight (continuous
 * batching); the result equals hasf_smooth on the same image.
 * *ticket receives an id.  Errors: HASF_EINVAL, HASF_EBUDGET (the job alone
 * exceeds the budget). */
int hasf_submit(hasf_ctx *ctx, const hasf_image *img, uint64_t *ticket);

/* Report a submitted job's state: *done = 1 and *status = its result code
 * once it has finished (the ticket is then forgotten), else *done = 0.
 * Errors: HASF_ENOTFOUND (unknown or already reported ticket). */
int hasf_poll(hasf_ctx *ctx, uint64_t ticket, int *done, int *status);

/* Cancel a submitted job that has not been launched yet: it will be reported
 * done with status HASF_ECANCELLED.  Errors: HASF_ENOTFOUND (unknown ticket),
 * HASF_EPENDING (the job is already on the device; it runs to completion). */
int hasf_cancel(hasf_ctx *ctx, uint64_t ticket);

/* Block until every submitted job has finished. */
int hasf_drain(hasf_ctx *ctx);

/* Context options (tuning and fault injection), applied to later calls.
 *   HASF_OPT_FORCE_GANG  (0/1): run every image in gang mode (planes in global
 *                        memory, several CTAs per image) even if it fits one CTA;
 *   HASF_OPT_GANG_CTAS   (>= 0): CTAs per gang image, 0 = automatic;
 *   HASF_OPT_ROUND_CAP   (>= 0): rounds allowed per priority level before the
 *                        device gives up with HASF_ETIMEOUT, 0 = automatic
 *                        (pixels + 2, never reached by a correct run);
 *   HASF_OPT_SERVE_STREAMS (1..16): concurrent batches of the server;
 *   HASF_OPT_SERVE_BATCH (1..4096): most jobs the server puts in one launch;
 *   HASF_OPT_STATS       (0/1): count the kernels' work (see hasf_read_stats);
 *   HASF_OPT_GENERIC_ONLY (0/1): run every image on the generic kernels (one
 *                        CTA with planes in shared memory, or a gang with planes
 *                        in L2) instead of the register and tiled kernels (the
 *                        result is the same; for comparisons);
 *   HASF_OPT_TILES       (0/1/2): images larger than 512 x 512 with rmax <= 31
 *                        run on the tiled register kernel -- 1 (default): as
 *                        thread-block clusters when they have at most 16 tiles
 *                        of 512 x 512, else as a gang; 2: always as a gang;
 *                        0: never (generic kernels);
 *   HASF_OPT_HOST_MAPPED (0/1/2): how hasf_smooth_host moves host buffers
 *                        the device can reach -- 2 (default): the register
 *                        kernel's images in place, the others as in 1;
 *                        1: page-locked mapped buffers through one launch of
 *                        the library's copy kernel per direction; 0: one copy
 *                        call per buffer;
 *   HASF_OPT_WAIT_DEADLINE_MS (0..60000): how long a CTA of a gang waits at
 *                        the gang barrier for the others before the job gives
 *                        up with HASF_ETIMEOUT, 0 = 4000 ms;
 *   HASF_OPT_FAULT_GANG_SKIP (0/1): fault injection for tests of the failure
 *                        path -- 1 makes CTA 0 of every gang of two or more
 *                        CTAs leave its job before its first barrier, as a CTA
 *                        that died would; the others' waits run out at the
 *                        deadline and the job reports HASF_ETIMEOUT (no device
 *                        fault; the context stays usable); 0 = off;
 *   HASF_OPT_FAULT_ALLOC (>= 0): fault injection -- the n-th device or pinned
 *                        host allocation the context makes from now on fails
 *                        as if the memory were exhausted (the call returns
 *                        HASF_ENOMEM); 0 = off;
 *   HASF_OPT_ROW_GROUP   (0, 1, 2 or 4): the single-tile register kernel's sweep
 *                        schedule -- how many rows of one parity a thread tests
 *                        together (sharing their neighbour rows, one warp vote
 *                        and one shuffle round); 0 (default) = the autotuner's
 *                        choice for the image's size bucket, else 4.  The result
 *                        is the same for every schedule.
 *   HASF_OPT_SIMPLE3_TABLE (0/1): hasf_smooth3d's simple-voxel test -- 1
 *                        (default): one read of a table of all 2^26
 *                        neighbourhoods (8 MB of device memory, built by the
 *                        context's first volume call from the flood-fill test
 *                        and kept until hasf_destroy); 0: the flood fills of
 *                        the neighbourhood in every test.  The same result.
 * Errors: HASF_EINVAL for an unknown option or value. */
enum {
    HASF_OPT_FORCE_GANG = 1,
    HASF_OPT_GANG_CTAS = 2,
    HASF_OPT_ROUND_CAP = 3,
    HASF_OPT_SERVE_STREAMS = 4,
    HASF_OPT_SERVE_BATCH = 5,
    HASF_OPT_STATS = 6,
    HASF_OPT_GENERIC_ONLY = 7,
    HASF_OPT_TILES = 8,
    HASF_OPT_HOST_MAPPED = 9,
    HASF_OPT_WAIT_DEADLINE_MS = 10,
    HASF_OPT_FAULT_GANG_SKIP = 11,
    HASF_OPT_FAULT_ALLOC = 12,
    HASF_OPT_ROW_GROUP = 13,
    HASF_OPT_SIMPLE3_TABLE = 14
};
int hasf_set_option(hasf_ctx *ctx, int option, int64_t value);

/* Work counters accumulated by launches made while HASF_OPT_STATS was 1,
 * summed over images: [0] sweep word tests (32-pixel words tested, each word
 * counted once per subfield: the register kernel counts the rows of the groups
 * it tests, the other kernels every word of the rows they sweep), [1] shifted
 * feature words read by level updates,
 * [2] subfield passes, [3] priority levels that activated points, [4] rounds,
 * and [5] the number of kernel launches the context issued since the last
 * read (counted on the host whatever HASF_OPT_STATS is).  Synchronises the
 * device, copies the first n (1..6) counters to the HOST array out and resets
 * them.  Errors: HASF_EINVAL, HASF_ECUDA. */
int hasf_read_stats(hasf_ctx *ctx, uint64_t *out, int n);

/* Static description of a status code. */
const char *hasf_strerror(int status);

/* ---- CUDA graphs ---------------------------------------------------------------
 * Capture one batched launch of n images into a CUDA graph, for callers that
 * smooth new contents of the same buffers again and again (video, tiles of a
 * scan).  The descriptors -- pointers, sizes, rmax, connectivity -- are fixed
 * when the graph is made; the image bytes are read when it is launched.  The
 * graph owns its scratch memory (counted against the context's budget) and
 * must be destroyed before the context.  Errors as hasf_smooth_batch. */
typedef struct hasf_graph hasf_graph;
int hasf_graph_create(hasf_ctx *ctx, const hasf_image *imgs, int n, hasf_graph **graph);
/* Launch the captured work on `stream` (asynchronous). */
int hasf_graph_launch(hasf_graph *graph, void *stream);
/* Wait for the graph's launches and free it. */
int hasf_graph_destroy(hasf_graph *graph);

/* ---- Autotuner --------------------------------------------------------------
 * Images that do not fit the single-tile register kernel can run on the tiled
 * register kernel (one CTA per 512 x 512 tile), on the generic shared-memory
 * kernel (one CTA), or on the generic gang (several CTAs sharing planes in L2).
 * hasf_autotune times these candidates -- tiled when eligible, one-CTA when
 * the image fits it, and gangs of 1, 2, 4, ... CTAs -- on a synthetic image of
 * the given size, in batches that fill the GPU (throughput, the batched use),
 * and records the fastest for the size bucket (powers of two of width and
 * height, and rmax).  For images the single-tile register kernel takes it
 * times that kernel's sweep schedules instead (1, 2 or 4 rows tested
 * together, see HASF_OPT_ROW_GROUP) and records the fastest.  Later batches
 * use the recorded choices.  *ctas receives the CTAs per image: -1 = tiled,
 * 0 = one-CTA generic, g > 0 = gang of g CTAs (and 0 for images the
 * single-tile kernel takes).  Synchronous. */
int hasf_autotune(hasf_ctx *ctx, int32_t width, int32_t height, int32_t rmax,
                  int32_t connectivity, int32_t *ctas);
/* The choice recorded for the size bucket of (width, height, rmax): *ctas as
 * for hasf_autotune and *rows_per_group the register kernel's sweep schedule
 * (1, 2 or 4; 0 for images that kernel does not take).  Errors: HASF_EINVAL,
 * HASF_ENOTFOUND (nothing recorded for the bucket). */
int hasf_tuning_get(hasf_ctx *ctx, int32_t width, int32_t height, int32_t rmax,
                    int32_t *ctas, int32_t *rows_per_group);
/* Save / load the tuned choices as text ("log2w log2h rmax ctas group" lines;
 * group 0 = a choice of CTAs per image, 1/2/4 = a register-kernel schedule;
 * lines of four fields are read as group 0). */
int hasf_tuning_save(hasf_ctx *ctx, const char *path);
int hasf_tuning_load(hasf_ctx *ctx, const char *path);

/* ---- Volumes ---------------------------------------------------------------- */

/* One volume for the 3D filter: dense w x h x d bytes, x fastest (voxel
 * (x, y, z) at in[(z * height + y) * width + x]), non-zero = object; C, D
 * (same layout, may be NULL) as in hasf_image.  width, height, depth in
 * [1, 4096] with at most 2^31 voxels; rmax in [1, 12]. */
typedef struct hasf_volume {
    const uint8_t *in;
    uint8_t *out;         /* may equal in */
    const uint8_t *C;
    const uint8_t *D;
    int32_t width;
    int32_t height;
    int32_t depth;
    int32_t rmax;
    int32_t reserved[2];  /* must be 0 */
} hasf_volume;

/* HASF_rmax^{C,D} of n volumes (device pointers), asynchronously on `stream`.
 * The paper states the filter for 2D images and notes (Sec. 1) that it
 * carries over to 3D; this is that extension with (26, 6) adjacency: a voxel
 * is simple when its object 26-neighbours form one 26-connected component and
 * the background voxels of its 18-neighbourhood 6-connected to a face
 * neighbour form one 6-connected component; B_r is the ball |v|^2 <= r^2; the
 * sweep order is levels, then rounds of the eight subfields (x, y, z mod 2)
 * in the order s = 0..7 with parities (s & 1, (s >> 1) & 1, s >> 2).  Each
 * volume is processed by a gang of CTAs; the library owns the scratch (seven
 * bit planes per volume).  Errors as hasf_smooth_batch; a device-side
 * HASF_ETIMEOUT is reported by hasf_status_of. */
int hasf_smooth3d(hasf_ctx *ctx, const hasf_volume *vols, int n, void *stream);

/* ---- Single operators (the same kernels, one step of the filter) --------- */

/* Exact squared Euclidean distance transform (Sec. 4.1, Meijster's two
 * phases: per-column vertical distance, then per-row lower envelope of
 * parabolas).  feat: device uint8 image (width x height, row pitch `pitch`
 * bytes), non-zero = feature point.  If outside_is_feature is non-zero every
 * point outside the box is a feature too.  d: device int32 array of
 * width*height values (row-major, no padding) receiving the squared distance,
 * or -1 where there is no feature at all.  width, height in [1, 32768].
 * Asynchronous on `stream`; scratch comes from the context. */
int hasf_edt(hasf_ctx *ctx, const uint8_t *feat, int32_t width, int32_t height,
             int32_t pitch, int32_t outside_is_feature, int32_t *d, void *stream);

/* One operator of the filter on one image, asynchronously on `stream`:
 *   op 1: H(Z, W)   -- img->in = Z, img->C = W (NULL = empty); ultimate
 *                      thinning over priority levels 1..r^2 (points whose
 *                      priority exceeds r^2 are never removed);
 *   op 2: *H(Y, V)  -- img->in = Y, img->C = V (required); thickening over
 *                      levels 1..r^2;
 *   op 3: HC_r^C    -- img->C as for hasf_smooth;
 *   op 4: HF_r^D    -- img->D as for hasf_smooth;
 * with r = img->rmax.  Errors as hasf_smooth. */
int hasf_operator(hasf_ctx *ctx, int op, const hasf_image *img, void *stream);

/* Evaluate, on the device, the simple-point test the kernels use on all 256
 * neighbour codes (bit k = neighbour k in the order E, NE, N, NW, W, SW, S,
 * SE; y grows downward).  out256: HOST array receiving 0/1.  Synchronous. */
int hasf_simple_table(hasf_ctx *ctx, int32_t connectivity, uint8_t *out256);

/* The simple-voxel table hasf_smooth3d reads (HASF_OPT_SIMPLE3_TABLE 1), for
 * checking it: built on `stream` if the context has none yet (waited for),
 * then copied asynchronously on `stream` into the DEVICE array out of 2^21
 * uint32 words.  Bit i of the table (bit i % 32 of word i / 32) is 1 when the
 * centre voxel is simple ((26, 6) adjacency) in the 3 x 3 x 3 neighbourhood
 * whose 26 neighbours are the bits of i: the 27-bit position code
 * (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) with the centre, bit 13, taken out
 * (code bits 0..12 are bits 0..12 of i, code bits 14..26 are bits 13..25).
 * Errors: HASF_EINVAL for a null argument, HASF_ENOMEM, HASF_ECUDA. */
int hasf_simple3_table(hasf_ctx *ctx, uint32_t *out, void *stream);

/* Priority levels as the fused kernel derives them, for checking it: for
 * every pixel of the width x height device image `feat` (pitch bytes), the
 * smallest level l in {sums of two squares <= r^2} such that a point of the
 * feature set lies within squared distance l, else r^2 + 1.  The feature set
 * is, by `mode`: 0 = the object pixels of feat (a thickening's priority),
 * 1 = those plus every point outside the box, 2 = the background pixels of
 * feat plus every point outside the box (a thinning's priority).
 * d: device int32, width*height values, row-major.  r in [1, 64]. */
int hasf_levels(hasf_ctx *ctx, const uint8_t *feat, int32_t width, int32_t height,
                int32_t pitch, int32_t mode, int32_t r, int32_t *d, void *stream);

/* ---- Allocation-free form ---------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: latency-critical loops that must not
 * stall on cudaMalloc (which can synchronise the device), and code inside a
 * host framework or plug-in whose device memory belongs to that framework's
 * allocator.  It smooths one image like hasf_smooth, asynchronously on
 * `stream`, with no context, in one launch of one CTA: the register kernel of
 * hasf_smooth for images of at most 512 x 512 with rmax <= 31, else the fused
 * kernel with its bit planes in shared memory.  The kernels' scratch (an input
 * snapshot and the packed C and D planes) lives in a fixed array inside the
 * library (about 240 KB, held on every GPU that loads the library until the
 * process exits).  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Limit: height * ceil(width / 32) <= 20480 and the image's three bit planes
 * must fit one CTA's shared memory (about 1130 rows at 512 columns, 560 rows at
 * 1024 columns); larger images return HASF_EBUDGET.  rmax must lie in
 * [1, 64]: the run to stability that hasf_smooth offers for rmax < 0 is not
 * available here (it needs one more plane), and such an rmax returns
 * HASF_EINVAL, like the other argument errors of hasf_smooth.
 *
 * `status` is an optional DEVICE int: it is cleared on `stream` and then
 * receives 0, or HASF_ETIMEOUT if the device iteration cap was hit (NULL: the
 * status is kept inside the library and not reported).
 *
 * The first call on each device (with that device current) does a one-time
 * set-up: it loads the constant level table and looks up the device address of
 * the scratch array.  Make that first call before any stream capture.
 * All calls on one GPU share that GPU's copy of the array, which keeps the last
 * call's contents: calls that overlap on the GPU (for example on two streams)
 * race and corrupt each other's results; order them on one stream. */
int hasf_smooth_noalloc(const hasf_image *img, int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HASF_H_ */
