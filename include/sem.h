/*
 * sem.h -- C ABI of libsem, the GB300 (sm_103a) library for the in situ render path of
 * spectral-element (SEM) velocity fields: spectral derivative -> Q-criterion -> marching-cubes
 * isosurface -> z-buffer raster.
 *
 * Where the operations come from.  The paper instruments NekRS, a spectral-element code
 * (Sec. 1), so that fields resident in GPU memory are rendered to images every n time steps
 * (Sec. 3.1, Listing 1: an analysis with frequency="100"; Sec. 4.1: images every 100 steps
 * instead of checkpoints).  Its bridge is called once to initialise with the solver's data
 * and then once per step (Sec. 3.2, Listing 3), and its DataAdaptor hands over the mesh and
 * the field arrays (Sec. 3.2, Listing 2: GetMesh / AddArray).  The paper does this on the CPU
 * after a device-to-host copy (Sec. 3.2) through third-party renderers; it does not define
 * the visualisation arithmetic.  This library keeps the data on the device and states that
 * arithmetic from textbook definitions, cited per call below.  sem_create/sem_load_mesh play
 * the role of the bridge's initialise + GetMesh; sem_qcriterion/sem_isosurface/sem_render
 * are the per-step analysis.
 *
 * Conventions (all calls):
 *   - Element e of order N has (N+1)^3 Gauss-Lobatto-Legendre (GLL) nodes ordered
 *     n = i + (N+1)(j + (N+1)k) (r fastest); a field is float f[E][(N+1)^3] (element-major,
 *     the Nek layout), one array per component.
 *   - Device pointers are CUDA device pointers of the context's device and must be 16-byte
 *     aligned, else SEM_ERR_ARG; triangle buffers (tris, tri_elem) need only 4-byte alignment,
 *     so several isosurfaces can be written back to back into one buffer.  The caller owns every field, triangle and image buffer; the
 *     library owns sem_ctx, sem_mesh and its own scratch memory.
 *   - Every call is stream-ordered on the context's stream and returns without waiting,
 *     except where a call states that it synchronises.  Kernel-side failures that are only
 *     visible later (a bounded wait that ran out) are reported by sem_synchronize.
 *   - No call throws, aborts or falls back to the CPU.  On failure a call returns a nonzero
 *     sem_status, writes no output past the stated bounds, and sem_last_error(ctx) describes
 *     the failure.
 *   - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>

#if defined(__GNUC__)
#define SEM_API __attribute__((visibility("default")))
#else
#define SEM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem_ctx sem_ctx;   /* opaque: device, stream, scratch, error text        */
typedef struct sem_mesh sem_mesh; /* opaque: per-element affine boxes + GLL tables      */

typedef enum {
    SEM_OK = 0,
    SEM_ERR_ARG = 1,          /* bad pointer, size, alignment, order N or precision       */
    SEM_ERR_CAPACITY = 2,     /* output buffer too small; the required size is returned   */
    SEM_ERR_OOM = 3,          /* device scratch allocation failed                         */
    SEM_ERR_CUDA = 4,         /* a CUDA runtime call failed                               */
    SEM_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out (kernel returned)     */
    SEM_ERR_UNSUPPORTED = 6   /* valid request this build does not implement (e.g. a
                                 curved mesh, an unimplemented precision)                 */
} sem_status;

/* Arithmetic of the derivative contraction (sem_derivatives, sem_qcriterion). */
typedef enum {
    SEM_FP32 = 0,   /* FP32 FFMA (the plain path)                                            */
    SEM_TF32 = 1,   /* tensor cores, TF32 operands, FP32 accumulation                        */
    SEM_FP16 = 2,   /* tensor cores, FP16 operands, FP32 accumulation                        */
    SEM_BF16 = 3,   /* tensor cores, BF16 operands, FP32 accumulation                        */
    SEM_BF16X2 = 4  /* tensor cores, operands split into BF16 hi + lo, FP32 accumulation      */
} sem_prec;

/* Largest polynomial order accepted by sem_load_mesh. */
#define SEM_MAX_ORDER 15
/* Triangle slots per marching-cubes case in sem_mc_table. */
#define SEM_MC_MAXT 12
/* Most isovalues one sem_isosurface_multi call extracts. */
#define SEM_MAX_ISO 8
/* Most further fields one sem_qcriterion_isosurface_fields_async call extracts. */
#define SEM_MAX_FIELDS 4

/* Camera of sem_render.  View basis f = unit(center-eye), s = unit(f x up), u = s x f;
 * view coordinates xv = s.(p-eye), yv = u.(p-eye), zv = f.(p-eye).
 *   ortho != 0: x_ndc = xv/(half_h*W/H), y_ndc = yv/half_h, depth = (zv-znear)/(zfar-znear)
 *   ortho == 0: x_ndc = xv/(zv*tan(fovy/2)*W/H), y_ndc = yv/(zv*tan(fovy/2)),
 *               depth = zfar/(zfar-znear) * (1 - znear/zv)
 * screen x = (x_ndc+1)/2*W, y = (1-y_ndc)/2*H (row 0 at the top). */
typedef struct {
    int32_t ortho;
    float eye[3];
    float center[3];
    float up[3];
    float fovy_deg;
    float half_h;
    float znear;
    float zfar;
} sem_camera;

/* ABI version of this header (bumped on any signature change). */
SEM_API int sem_version(void);

/* Create a context on CUDA device `device` that issues all work on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Uploads the constant tables (GLL, marching cubes).
 * Synchronous.  *out is NULL on failure. */
SEM_API sem_status sem_create(int device, void *stream, sem_ctx **out);

/* Destroy a context (waits for its stream, frees its scratch).  NULL is a no-op. */
SEM_API void sem_destroy(sem_ctx *ctx);

/* Text of the last failure on this context ("" if none).  Owned by the context; valid until
 * the next call on it.  With ctx == NULL, the last failure of sem_create on this thread. */
SEM_API const char *sem_last_error(const sem_ctx *ctx);

/* Switch the context to another stream of the same device. */
SEM_API sem_status sem_set_stream(sem_ctx *ctx, void *stream);

/* Wait for the context's stream; report any device-side failure flagged since the last call
 * (SEM_ERR_TIMEOUT) and clear it. */
SEM_API sem_status sem_synchronize(sem_ctx *ctx);

/* Failure-detection test hook (no counterpart in the paper).  The Q kernels of
 * sem_qcriterion, sem_qcriterion_batch and sem_derivatives (FP32 path) wait on an mbarrier for
 * each stage's input copies; every such wait gives up after a bounded number of polls, records
 * SEM_ERR_TIMEOUT on the context's device flag, waits (with the default limit) for its copies
 * still in flight and returns, leaving the outputs incomplete.  This call sets that limit for
 * later launches on ctx: polls >= 0 (0 = give up at the first wait, so the timeout path runs
 * deterministically), polls < 0 restores the default (about 2^24 polls, seconds).  Host only;
 * takes effect at the next launch. */
SEM_API sem_status sem_debug_set_wait_limit(sem_ctx *ctx, int64_t polls);

/* Device memory the library holds for ctx (scratch arenas, tables, meshes loaded with ctx,
 * autoencoders created on ctx; caller-owned buffers are not counted): *in_use now and *peak,
 * the high-water mark since sem_create.  Free meshes and autoencoders before their context. */
SEM_API sem_status sem_memory(sem_ctx *ctx, int64_t *in_use, int64_t *peak);

/* Kernel trace (instrumentation; no counterpart in the paper).  While on, every kernel the
 * library launches on the context's stream outside a stream capture is bracketed by a pair of
 * CUDA events on that stream.  sem_trace_collect waits for the recorded launches, sums their
 * device time per kernel name (in first-launch order) and returns the number of kernels in
 * *n_kernels; sem_trace_entry reads entry k: *name (a static string owned by the library),
 * the summed milliseconds and the launch count.  Collecting clears the record.  Tracing adds
 * two event records per launch and is off by default. */
SEM_API sem_status sem_trace_enable(sem_ctx *ctx, int on);
SEM_API sem_status sem_trace_collect(sem_ctx *ctx, int *n_kernels);
SEM_API sem_status sem_trace_entry(sem_ctx *ctx, int k, const char **name, double *total_ms, int64_t *launches);

/* Load a mesh of E hexahedral elements of order N (1 <= N <= SEM_MAX_ORDER).
 * xyz_host: HOST array of 3*E*(N+1)^3 doubles, SoA x | y | z, node order as above; copied.
 * When every element is an axis-aligned affine box (x depends only on i, y on j, z on k, with
 * the GLL spacing, x = x0 + (xi+1)/2 (x1-x0)), the mesh keeps six numbers per element and the
 * derivative uses the per-axis factors 2/(x1-x0).  Otherwise the mesh is general (curved): the
 * library computes at every node, in FP64 on the host, the Jacobian d x_c / d r_d of the
 * isoparametric map (D applied to the node coordinates) and keeps its inverse d r_d / d x_j
 * (9 floats per node) and the node coordinates (3 floats per node) on the device; derivatives
 * then follow the chain rule d u / d x_j = sum_d (d u / d r_d)(d r_d / d x_j) (Deville, Fischer
 * & Mund, Sec. 4.5) and isosurface vertices lie between the nodes' own coordinates.  On general
 * meshes the tensor-core precisions, sem_qcriterion_batch and sem_isosurface_noalloc return
 * SEM_ERR_UNSUPPORTED.  Errors: SEM_ERR_ARG for a non-finite coordinate or a node whose Jacobian
 * determinant is not positive (an inverted or degenerate element).  Synchronous; the general
 * case costs O(E (N+1)^4) host work.  Free with sem_mesh_free. */
SEM_API sem_status sem_load_mesh(sem_ctx *ctx, int N, int64_t E, const double *xyz_host, sem_mesh **out);
SEM_API void sem_mesh_free(sem_mesh *mesh);
SEM_API sem_status sem_mesh_info(const sem_mesh *mesh, int *N, int64_t *E);

/* Spectral derivative of one field u (device, E*(N+1)^3 floats):
 *   du/dr[k][j][i] = sum_m D[i][m] u[k][j][m]  (likewise s over j, t over k),
 *   du/dx = 2/(x1-x0) du/dr, du/dy = 2/(y1-y0) du/ds, du/dz = 2/(z1-z0) du/dt on box meshes,
 *   du/dx_j = sum_d du/dr_d dr_d/dx_j on general meshes (see sem_load_mesh),
 * with D the GLL collocation derivative matrix (Canuto et al., Spectral Methods, Sec. 2.3).
 * Derivatives are element-local (no averaging across element faces).
 * dudx, dudy, dudz: device, E*(N+1)^3 floats each, must not alias u. */
SEM_API sem_status sem_derivatives(sem_ctx *ctx, const sem_mesh *mesh, const float *u, float *dudx,
                           float *dudy, float *dudz, sem_prec prec);

/* Q-criterion (Hunt, Wray & Moin 1988) of the velocity (u, v, w) at every node:
 *   J_ij = du_i/dx_j (as in sem_derivatives),  Q = 1/2(|Omega|^2 - |S|^2) = -1/2 sum_ij J_ij J_ji.
 * u, v, w, Q: device, E*(N+1)^3 floats each; Q must not alias the inputs.
 * prec: SEM_FP32 at every order; SEM_TF32, SEM_FP16, SEM_BF16 and SEM_BF16X2 run the s- and
 * t-contractions on the tensor cores (the r-contraction and Q stay FP32) and exist for N = 7
 * only (SEM_ERR_UNSUPPORTED otherwise). */
SEM_API sem_status sem_qcriterion(sem_ctx *ctx, const sem_mesh *mesh, const float *u, const float *v,
                          const float *w, float *Q, sem_prec prec);

/* Q of n partitions in as few launches as possible (the batched form of sem_qcriterion, FP32):
 * meshes[p] with fields u[p], v[p], w[p] -> Q[p] (device pointers, each as in sem_qcriterion;
 * the pointer arrays are HOST arrays).  Partitions of one order share one persistent launch
 * (up to 48 per launch), whatever their element counts; orders may be mixed.  Results equal
 * sem_qcriterion's on each partition bit for bit.  Asynchronous; may be captured in a graph. */
SEM_API sem_status sem_qcriterion_batch(sem_ctx *ctx, int n, const sem_mesh *const *meshes, const float *const *u,
                                        const float *const *v, const float *const *w, float *const *Q);

/* Marching-cubes isosurface (Lorensen & Cline 1987) of f = iso over the N^3 sub-hexes of each
 * element's GLL lattice.  Cell (i,j,k), corner v = a + 2b + 4c at node (i+a, j+b, k+c);
 * case = sum_v [f_v >= iso] 2^v (NaN counts as below).  The case table is the library's own,
 * generated from a face-consistent rule (see sem_mc_table); the surface is crack-free across
 * cells and elements and its normals (p1-p0)x(p2-p0) point toward increasing f.
 * Cut edge (lo, hi), lo the lower corner: t = (iso - f_lo)/(f_hi - f_lo),
 * p = p_lo + t (p_hi - p_lo).  Triangles are written in (element, cell i + N(j + Nk), table)
 * order as float tris[ntri][3][3] (vertex-major xyz) with tri_elem[ntri] = element index.
 *   f:        device, E*(N+1)^3 floats
 *   tris:     device, cap*9 floats, or NULL to only count (then cap is ignored, nothing
 *             but *ntri_out and cases is written, and the call returns SEM_OK)
 *   tri_elem: device, cap int32 (may be NULL)
 *   cap:      capacity in triangles (>= 0)
 *   ntri_out: HOST; receives the triangle count
 *   cases:    device, E*N^3 bytes, or NULL; receives every cell's case index
 * Synchronises once (to read the count back).  If the count exceeds cap, returns
 * SEM_ERR_CAPACITY with *ntri_out = the required count and writes no triangle. */
SEM_API sem_status sem_isosurface(sem_ctx *ctx, const sem_mesh *mesh, const float *f, float iso, float *tris,
                          int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases);

/* sem_isosurface for several isovalues of one field at once (1 <= niso <= SEM_MAX_ISO).  The
 * result equals niso sem_isosurface calls written back to back: the triangles of isovalue q
 * follow those of isovalue q-1, each in (element, cell, table) order, and ntri_out[q] (HOST,
 * niso entries) receives isovalue q's count.  The field is read once per pass for all
 * isovalues, and the call synchronises once.  cases (device, niso*E*N^3 bytes, or NULL) is laid
 * out [q][e][cell].  tris NULL: count only.  If the total exceeds cap, returns
 * SEM_ERR_CAPACITY with ntri_out filled and writes no triangle. */
SEM_API sem_status sem_isosurface_multi(sem_ctx *ctx, const sem_mesh *mesh, const float *f, const float *isos_host,
                                        int niso, float *tris, int32_t *tri_elem, int64_t cap, int64_t *ntri_out,
                                        uint8_t *cases);

/* sem_isosurface_multi without host synchronisation, for work captured in a CUDA graph.
 * counts_dev: device int64[niso + 1] receives the segment starts (counts_dev[q] = first triangle
 * of isovalue q, counts_dev[niso] = total).  If the total exceeds cap, no triangle is written and
 * the context's device flag records SEM_ERR_CAPACITY (reported by sem_synchronize); counts_dev
 * still holds the required sizes.  The library's scratch must already be large enough when the
 * stream is being captured: make one uncaptured call with the same mesh and niso first
 * (otherwise SEM_ERR_CAPACITY, nothing launched).  Other arguments as sem_isosurface_multi. */
SEM_API sem_status sem_isosurface_multi_async(sem_ctx *ctx, const sem_mesh *mesh, const float *f,
                                              const float *isos_host, int niso, float *tris, int32_t *tri_elem,
                                              int64_t cap, int64_t *counts_dev, uint8_t *cases);

/* sem_qcriterion (FP32) followed by sem_isosurface_multi_async of Q at isos_host[0..niso-1], with
 * the isosurface pass's per-element triangle counting done by the Q kernel itself from the Q it
 * has just computed, so Q is not read back from memory for counting (on N = 7 box meshes; on other
 * meshes the two passes run one after the other).  Q, the triangles, counts_dev and every error
 * are exactly those of the two calls: Q and tris bit for bit.  No host synchronisation; may be
 * captured in a CUDA graph (scratch rule of sem_isosurface_multi_async).  u, v, w, Q: device,
 * E*(N+1)^3 floats each, Q not aliasing the inputs; other arguments as
 * sem_isosurface_multi_async (no per-cell cases). */
SEM_API sem_status sem_qcriterion_isosurface_async(sem_ctx *ctx, const sem_mesh *mesh, const float *u,
                                                   const float *v, const float *w, float *Q, const float *isos_host,
                                                   int niso, float *tris, int32_t *tri_elem, int64_t cap,
                                                   int64_t *counts_dev);

/* sem_isosurface_multi_async appending behind triangles already in `tris`, so that the
 * isosurfaces of several fields (e.g. Q and temperature) fill one buffer back to back and one
 * sem_render_async draws them as consecutive segments, all without host synchronisation.
 * counts_dev (device int64[niso + 1]) is read and written on the device: counts_dev[0] is an
 * INPUT, the index in tris of this call's first triangle (typically the last entry an earlier
 * sem_isosurface_multi_async or append call wrote, i.e. pass that call's counts_dev + its niso);
 * the call writes counts_dev[q] = counts_dev[0] + (triangles of isovalues 0..q-1) for
 * q = 1..niso.  cap is the capacity of the whole buffer from tris[0]; if counts_dev[0] plus this
 * call's total exceeds it, no triangle is written and the device flag records
 * SEM_ERR_CAPACITY (reported by sem_synchronize).  Triangle order and everything else as
 * sem_isosurface_multi_async (same scratch rule under stream capture). */
SEM_API sem_status sem_isosurface_multi_append_async(sem_ctx *ctx, const sem_mesh *mesh, const float *f,
                                                     const float *isos_host, int niso, float *tris,
                                                     int32_t *tri_elem, int64_t cap, int64_t *counts_dev,
                                                     uint8_t *cases);

/* Q of (u, v, w) with its isosurfaces, and the isosurfaces of nfields further fields of the same
 * mesh, into one triangle buffer in one call: the result of sem_qcriterion_isosurface_async(Q at
 * q_isos[0..q_niso-1]) followed, for k = 0..nfields-1, by sem_isosurface_multi_append_async of
 * fields[k] at its f_niso[k] isovalues (f_isos holds them back to back, field 0's first), each
 * appending behind the one before.  Q, tris, tri_elem and counts_dev are bit for bit those of that
 * call sequence.  counts_dev: device int64[1 + q_niso + sum f_niso] receives every segment start,
 * Q's isovalues first then the fields' in order, and the grand total last.
 * Concurrency: after the Q kernel, the further fields' passes (counting, scan, emit) run on an
 * auxiliary stream of the context, forked from and joined back to the context's stream within
 * the call, so they overlap Q's scan and emit; stream order as seen by the caller is unchanged,
 * and the whole call may be captured in a CUDA graph (scratch rule of sem_isosurface_multi_async).
 * While the context's emit autotuner (sem_autotune_set) still has to time a launch of this call,
 * or the kernel trace (sem_trace_enable) is on, the passes run one after the other on the
 * context's stream, so that each timing is the kernel's own; so they do when the call is
 * captured before any uncaptured call of it has created the auxiliary stream.  Each field keeps scratch of its own.  Arguments: fields: HOST array of nfields
 * device pointers (E*(N+1)^3 floats each); f_isos, f_niso: HOST; 0 <= nfields <= SEM_MAX_FIELDS,
 * 1 <= q_niso, f_niso[k] <= SEM_MAX_ISO; cap: capacity of the whole buffer; a total above it
 * writes no triangle of the segment that overflows (or of any later one) and raises
 * SEM_ERR_CAPACITY on the device flag.  Other arguments and errors as
 * sem_qcriterion_isosurface_async. */
SEM_API sem_status sem_qcriterion_isosurface_fields_async(sem_ctx *ctx, const sem_mesh *mesh, const float *u,
                                                          const float *v, const float *w, float *Q,
                                                          const float *q_isos, int q_niso, int nfields,
                                                          const float *const *fields, const float *f_isos,
                                                          const int *f_niso, float *tris, int32_t *tri_elem,
                                                          int64_t cap, int64_t *counts_dev);

/* One in situ frame in one call: sem_qcriterion_isosurface_fields_async (Q, its isosurfaces and
 * the further fields' isosurfaces into tris, segment starts into counts_dev) followed by
 * sem_render_async of all nseg = q_niso + sum f_niso segments (colours seg_rgb[3*nseg], HOST, or
 * NULL for the palette) into rgba/depth.  The frame is drawn in parts: each stream rasterises the
 * segments it has just emitted -- Q's on the context's stream, the further fields' on the
 * auxiliary stream -- into the same depth keys, and the large-triangle pass and the resolve run
 * once, after the join.  rgba, depth, Q, tris, tri_elem and counts_dev are bit for bit those of
 * the two calls.  With nfields = 0, and on the first call for a frame size while the context's
 * autotuner still has to choose the render's launch widths (so they are timed on a whole frame),
 * the call runs the two calls as such.  No host synchronisation; may be captured in a CUDA graph (scratch rule of
 * sem_isosurface_multi_async; render scratch likewise sized by an uncaptured call).  Arguments
 * and errors as the two calls (cap < 2^31, nseg <= 64); one frame in progress per context. */
SEM_API sem_status sem_frame_async(sem_ctx *ctx, const sem_mesh *mesh, const float *u, const float *v, const float *w,
                                   float *Q, const float *q_isos, int q_niso, int nfields, const float *const *fields,
                                   const float *f_isos, const int *f_niso, float *tris, int32_t *tri_elem,
                                   int64_t cap, int64_t *counts_dev, const float *seg_rgb, const sem_camera *cam,
                                   int W, int H, uint8_t *rgba, float *depth);

/* Largest mesh (in elements) that sem_isosurface_noalloc accepts. */
#define SEM_NOALLOC_MAX_ELEMENTS 262144

/* sem_isosurface without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory while they run -- for example
 * an in situ hook inside a solver's time step when the solver has already committed the GPU's
 * memory to its own fields and pools, so that a cudaMalloc would fail or stall the step.
 * sem_isosurface may grow the context's scratch arena with cudaMalloc/cudaFree; this variant
 * instead keeps its scratch (per-element counts, triangle offsets, scan partials, about 3 MB)
 * in one fixed device array inside the library, which every GPU that loads the library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Arguments, results, ordering, synchronisation and errors are those of sem_isosurface.
 *     The context and the mesh must have been created beforehand (sem_create and
 *     sem_load_mesh do allocate).
 *   - E may be at most SEM_NOALLOC_MAX_ELEMENTS; a larger mesh is rejected with SEM_ERR_ARG
 *     and a message naming the limit, and nothing is launched.
 *   - sem_create does this entry point's set-up on its device: it looks up the array's device
 *     address (cudaGetSymbolAddress; the host-side symbol is only a stand-in) and keeps it in
 *     the context, and it makes the runtime load the array and every kernel this entry point
 *     launches, so that under lazy module loading no call of it loads code or data (which
 *     would allocate).  A context created after a cudaDeviceReset looks the address up again;
 *     contexts that lived through a reset are invalid, as for every other call.
 *   - Every call on a device shares the one array and leaves its contents behind for the next
 *     call.  Calls whose work overlaps on the GPU (different streams or contexts, or several
 *     host threads) race on it and give wrong results: issue them one after another. */
SEM_API sem_status sem_isosurface_noalloc(sem_ctx *ctx, const sem_mesh *mesh, const float *f, float iso,
                                          float *tris, int32_t *tri_elem, int64_t cap, int64_t *ntri_out,
                                          uint8_t *cases);

/* Z-buffer raster of a triangle soup into a headless RGBA8 + depth image.
 * Triangles are coloured per contiguous segment: segment s holds seg_ntri[s] triangles and
 * colour seg_rgb[3s..3s+2] (HOST arrays; seg_rgb NULL = built-in palette).  Pixel (x, y)
 * samples (x+0.5, y+0.5); coverage uses edge functions with the top-left fill rule; zero-area
 * triangles and triangles with a vertex outside znear < zv < zfar are dropped; no back-face
 * culling.  Depth is interpolated in screen space; the smallest (depth, triangle index) wins,
 * so the image does not depend on execution order.  Flat headlight shading:
 * c = rgb * (0.15 + 0.85 |n.l|), n the face normal, l = -f; rgba8 = floor(clamp(c)*255 + .5),
 * alpha 255.  Background: rgba (0,0,0,0), depth 1.
 *   tris:  device, ntri*9 floats;  rgba: device, H*W*4 bytes;  depth: device, H*W floats (may
 *   be NULL).  nseg in [1, 16]; sum(seg_ntri) == ntri.
 * Synchronises once (to size the tile lists). */
SEM_API sem_status sem_render(sem_ctx *ctx, const float *tris, int64_t ntri, const int64_t *seg_ntri, int nseg,
                      const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba,
                      float *depth);

/* sem_render without host synchronisation, segments read from the device: seg_start_dev is a
 * device int64[nseg + 1] of segment starts (e.g. counts_dev of sem_isosurface_multi_async);
 * triangles [seg_start_dev[0], seg_start_dev[nseg]) are drawn, at most ntri_max (a HOST upper
 * bound that sizes the launch; tris must hold ntri_max triangles).  Scratch as in
 * sem_isosurface_multi_async: make one uncaptured call with the same W, H and ntri_max first. */
SEM_API sem_status sem_render_async(sem_ctx *ctx, const float *tris, int64_t ntri_max, const int64_t *seg_start_dev,
                                    int nseg, const float *seg_rgb, const sem_camera *cam, int W, int H,
                                    uint8_t *rgba, float *depth);

/* sem_render_async with up to 64 segments, of which only those whose bit is set in seg_mask
 * (bit s for segment s) are drawn, e.g. one isovalue out of the (partition, isovalue) segments
 * that several sem_isosurface_multi_async / _append_async calls wrote back to back.  Triangles of
 * segments not drawn neither cover pixels nor take part in the depth test; the frame equals
 * sem_render of the drawn segments' triangles alone with their indices unchanged (ties between
 * equal depths still go to the lower index).  nseg in [1, 64]; seg_rgb (HOST, 3 nseg floats, or
 * NULL = the built-in palette repeated every 16 segments).  Other arguments and rules as
 * sem_render_async. */
SEM_API sem_status sem_render_segments_async(sem_ctx *ctx, const float *tris, int64_t ntri_max,
                                             const int64_t *seg_start_dev, int nseg, const float *seg_rgb,
                                             uint64_t seg_mask, const sem_camera *cam, int W, int H, uint8_t *rgba,
                                             float *depth);

/* FP64 reductions of a triangle soup (device, ntri*9 floats): out_host[0] = total area
 * sum |(p1-p0)x(p2-p0)|/2, out_host[1] = enclosed volume sum p0.(p1 x p2)/6 (divergence
 * theorem; positive when normals point out of the enclosed region).  Synchronises. */
SEM_API sem_status sem_surface_measures(sem_ctx *ctx, const float *tris, int64_t ntri, double *out_host);

/* Largest value of a device float array (NaNs ignored), e.g. for iso = fraction * max Q.
 * Synchronises.  n >= 1. */
SEM_API sem_status sem_field_max(sem_ctx *ctx, const float *f, int64_t n, float *max_host);

/* ------------------------------------------------------------------------------------------
 * Learned per-element compression (no counterpart in the paper's code; its motivation is the
 * transfer volume of in-transit analysis, Sec. 4.2).  An MLP autoencoder per element of order
 * N = 7: the 3 x 512 nodal velocity values, normalised per component, go through
 *   encoder  H1 = X W1^T + b1, A1 = gelu(H1), Z = A1 W2^T + b2      1536 -> 512 -> 48
 *   decoder  H3 = Z W3^T + b3, A3 = gelu(H3), Y = A3 W4^T + b4      48 -> 512 -> 1536
 * with gelu(x) = x Phi(x) (exact erf form), loss = mean over all entries of (Y - X)^2 and
 * AdamW updates (Loshchilov & Hutter 2019, bias-corrected moments, weight decay decoupled:
 * w -= lr (mhat / (sqrt(vhat) + eps) + wd w)).  All products run on the tensor cores in BF16
 * with FP32 accumulation; weights are kept in FP32 and copied to BF16 after each update; the
 * latent Z is BF16 (48 values = 96 bytes per element, 64x fewer than 1536 FP32 values) and the
 * decoder and training graph see the BF16 latent (its gradient passes through the rounding).
 *
 * Parameter arrays on the host are FP32, flattened in the order W1 (512 x 1536, row-major),
 * b1 (512), W2 (48 x 512), b2 (48), W3 (512 x 48), b3 (512), W4 (1536 x 512), b4 (1536):
 * sem_ae_param_count() values.  A sample is one element's 1536 values [u(512) | v(512) |
 * w(512)] (node order i + 8 j + 64 k), FP32; training reads samples from a device array
 * samples[n][1536] at the rows a device int64 array idx[B] names (the caller draws them).
 * ------------------------------------------------------------------------------------------ */
typedef struct sem_ae sem_ae;

/* Number of FP32 values in the flattened parameter arrays (1,624,624). */
SEM_API int64_t sem_ae_param_count(void);

/* Create an autoencoder on ctx's device with all parameters zero, for training batches of at
 * most `batch` samples (a multiple of 128; encode/decode work in chunks of `batch`).
 * Allocates its parameters, Adam moments, gradients and activations (about 28 KB per batch
 * row plus 26 MB).  Free with sem_ae_destroy. */
SEM_API sem_status sem_ae_create(sem_ctx *ctx, int batch, sem_ae **out);
SEM_API void sem_ae_destroy(sem_ae *ae);

/* Parameters (and the Adam moments with the step count, for checkpoints) from/to HOST
 * arrays of sem_ae_param_count() FP32 values.  Synchronous. */
SEM_API sem_status sem_ae_set_params(sem_ae *ae, const float *host, int64_t n);
SEM_API sem_status sem_ae_get_params(sem_ae *ae, float *host, int64_t n);
SEM_API sem_status sem_ae_get_state(sem_ae *ae, float *m_host, float *v_host, int64_t n, int64_t *step);
SEM_API sem_status sem_ae_set_state(sem_ae *ae, const float *m_host, const float *v_host, int64_t n, int64_t step);

/* Normalisation X = (value - mean[c]) / std[c] per component c.  sem_ae_fit_normalization
 * takes per-component means and one common scale (root of the mean per-component variance)
 * over device samples[n][1536] (FP64 sums; synchronous). */
SEM_API sem_status sem_ae_set_normalization(sem_ae *ae, const float mean[3], const float stdv[3]);
SEM_API sem_status sem_ae_get_normalization(sem_ae *ae, float mean[3], float stdv[3]);
SEM_API sem_status sem_ae_fit_normalization(sem_ae *ae, const float *samples, int64_t n);

/* Loss and gradients for the batch samples[idx[0..B-1]] (samples: n_samples rows) without
 * updating: *loss_host = the mean squared error; grad_host (HOST, flattened like the
 * parameters, or NULL) the gradient.  1 <= B <= batch.  An index outside [0, n_samples) is
 * read as the component means and raises SEM_ERR_ARG on the device flag (reported by
 * sem_synchronize).  Synchronous. */
SEM_API sem_status sem_ae_loss_grad(sem_ae *ae, const float *samples, int64_t n_samples, const int64_t *idx, int B,
                                    float *loss_host, float *grad_host, int64_t n);

/* One AdamW training step on the batch samples[idx[0..B-1]] (indices checked as in
 * sem_ae_loss_grad; asynchronous on the context's
 * stream; may be captured in a CUDA graph once the step count is fixed by the caller).
 * loss_dev (device float, or NULL) receives the batch's SUM of squared errors (divide by
 * 1536 B for the mean).  Bias corrections use the object's step count (incremented here). */
SEM_API sem_status sem_ae_train_step(sem_ae *ae, const float *samples, int64_t n_samples, const int64_t *idx, int B,
                                     float lr, float beta1, float beta2, float eps, float weight_decay,
                                     float *loss_dev);

/* Encode E elements of the device fields u, v, w ([E][512] FP32 each) to the device latent
 * [E][48] (BF16 bit patterns, 16-byte aligned); decode a latent back to u, v, w (16-byte
 * aligned).  Asynchronous. */
SEM_API sem_status sem_ae_encode(sem_ae *ae, const float *u, const float *v, const float *w, int64_t E,
                                 uint16_t *latent);
SEM_API sem_status sem_ae_decode(sem_ae *ae, const uint16_t *latent, int64_t E, float *u, float *v, float *w);

/* Autotuner of the tensor-core GEMM (on by default).  The first product of a given (M, N, K,
 * epilogue) on a context runs every candidate on the call's own data -- tile width BN in
 * {64, 128, 256}, 3 or 4 pipeline stages; for BN <= 128 also a persistent form (one CTA per SM
 * walking the output tiles, two TMEM accumulators so that a tile's epilogue overlaps the next
 * tile's MMAs; the same products in the same order); and for FP32 weight gradients a K split in
 * {1, 2, 4, 8, 16, 32} (at least 4 K blocks per split) with an ordered reduction of the partial
 * sums -- and keeps the fastest (CUDA events); later products of that shape reuse it.  Under
 * stream capture, or when off, the default (BN 128 where N allows, 4 stages, no split, one tile
 * per CTA) runs.  sem_autotune_set(ctx, 0) turns tuning off and forgets the choices;
 * sem_autotune_entry reads choice k (SEM_ERR_ARG past the last one), with the winner's time in
 * milliseconds; `persistent` (may be NULL) receives 1 for the persistent form. */
SEM_API sem_status sem_autotune_set(sem_ctx *ctx, int on);

/* The same switch tunes the launch of the isosurface emit pass (sem_isosurface,
 * sem_isosurface_multi and their asynchronous forms): the first emitting call of a given
 * (order N, element count E, isovalue count) runs the persistent emit kernel with 1, 2, 4 and 8
 * (element, isovalue) units per work-counter atomic (units that hold triangles: the scan before
 * the emit pass lists them), each once untimed and three times timed (its fastest run counts), keeps
 * the fastest and reuses it afterwards.  That first call waits for the GPU once.  Every
 * candidate writes the same triangles, so results do not depend on tuning.  Under stream
 * capture, or when off, 1 unit per atomic.  sem_autotune_emit_entry reads choice k
 * (SEM_ERR_ARG past the last one): N, E, isovalues, units per atomic and the winner's time in
 * milliseconds. */
SEM_API sem_status sem_autotune_emit_entry(sem_ctx *ctx, int k, int *N, int64_t *E, int *niso, int *units,
                                           float *ms);
/* The same switch tunes launch widths whose choice does not change any result: the persistent Q
 * kernels' CTAs per SM (so the elements each CTA walks through; kind 1: the N = 7 Q kernel,
 * 2: the N = 7 Q kernel with triangle counting, 3: other orders' Q, 4: other orders'
 * derivatives), chosen per (kind, order N, elements) among 1 .. the resident maximum; and the
 * grids of the render's large-triangle and resolve passes (kind 5, N = W, size = H), chosen per
 * frame size among five (large, resolve) pairs of CTAs per SM, width 0..4 = (6, 8), (4, 4),
 * (8, 16), (2, 8), (6, 2).  The first call of a key with tuning on, outside stream capture and
 * tracing, runs every candidate (once untimed, then three timed runs, the fastest counting) and
 * keeps the fastest; the others use
 * the widest Q launch and pair 0.  sem_autotune_width_entry reads choice k (SEM_ERR_ARG past the
 * last one). */
SEM_API sem_status sem_autotune_width_entry(sem_ctx *ctx, int k, int *kind, int *N, int64_t *size, int *width,
                                            float *ms);
SEM_API sem_status sem_autotune_entry(sem_ctx *ctx, int k, int64_t *M, int *N, int *K, int *mode, int *bn,
                                      int *stages, int *split, int *persistent, float *ms);

/* The library's tensor-core GEMM: C[M][N] = A[M][K] B[N][K]^T, A and B row-major BF16 bit
 * patterns (device, 16-byte aligned), C FP32 (device).  M % 128 == 0, N % 64 == 0,
 * K % 64 == 0 (else SEM_ERR_ARG).  FP32 accumulation.  Asynchronous. */
SEM_API sem_status sem_gemm_bf16(sem_ctx *ctx, const uint16_t *A, const uint16_t *B, int64_t M, int N, int K,
                                 float *C);

/* Host-only queries (no device needed). */

/* The library's marching-cubes case table: ntri[256] triangles per case and
 * edges[256][SEM_MC_MAXT][3] edge indices (-1 padded), edges numbered in lexicographic order
 * of their (lower, upper) corner pair.  Returns the largest ntri, or a negative value if the
 * generator failed. */
SEM_API int sem_mc_table(int32_t *ntri, int8_t *edges);

/* The library's GLL nodes xi[N+1] and derivative matrix D[(N+1)*(N+1)] (row-major, D[i][j] =
 * l_j'(xi_i)) in FP64, as computed for the device tables (which round them to FP32). */
SEM_API sem_status sem_gll(int N, double *xi, double *D);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
