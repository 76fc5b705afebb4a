// sem_internal.cuh -- shared internals of libsem (context, mesh, device helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sem.h"

#define SEM_WAIT_LIMIT (1ll << 24)   // bounded spin on an mbarrier phase (~ seconds)

// ------------------------------------------------------------------------------------------
// Host-side objects

struct RenderFrame;  // a frame drawn in parts (sem_render.cu)

// scratch arenas (each call uses its own so calls never overlap in scratch); SCR_ISO_F0 + k
// holds the isosurface pass of further field k of sem_qcriterion_isosurface_fields_async, which
// runs on the auxiliary stream while Q's pass (SCR_ISO) runs on the context's stream
enum { SCR_ISO = 0, SCR_RENDER = 1, SCR_MISC = 2, SCR_TRI = 3, SCR_ISO_F0 = 4, SCR_COUNT = 4 + SEM_MAX_FIELDS };

struct sem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int sm_count = 0;
    // device error word: kernels with bounded waits OR a code in here (SEM_ERR_TIMEOUT ...)
    int *d_flag = nullptr;
    // iteration limit of the Q kernels' waits for their input copies (sem_debug_set_wait_limit);
    // the waits that drain copies still in flight after an abort keep SEM_WAIT_LIMIT
    long long wait_limit = SEM_WAIT_LIMIT;
    // device address of sem_isosurface_noalloc's fixed scratch array on this device (resolved
    // by sem_create, so a context made after a device reset looks it up again)
    void *noalloc_scratch = nullptr;
    // device address of the case table's triangle counts (256 bytes), for kernels outside the
    // isosurface unit that classify cells
    const uint8_t *d_ntri = nullptr;
    // pinned host words for small read-backs (counts, totals)
    int64_t *h_pinned = nullptr;   // 16 int64 slots
    double *h_pinned_d = nullptr;  // 4 double slots
    // grow-only device scratch arenas
    void *scratch[SCR_COUNT] = {};
    size_t scratch_bytes[SCR_COUNT] = {};
    // auxiliary stream and the events that fork it from `stream` and join it back (created on
    // first use by sem_qcriterion_isosurface_fields_async)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_qseg = nullptr, ev_join = nullptr;
    // the frame sem_frame_async draws in parts (created on first use)
    RenderFrame *frame = nullptr;
    // the render key buffer must read "empty" (all ones) at the start of a frame
    bool render_keys_dirty = true;
    // tensor-core operand A (the stacked derivative matrices) per 16-bit type: 0 BF16, 1 FP16
    void *tc_A[3] = {nullptr, nullptr, nullptr};  // tensor-core D tables: bf16, fp16, tf32
    // autotuner: tile shape chosen per (M, N, K, epilogue) of the tensor-core GEMM
    bool autotune = true;
    struct GemmTune {
        int64_t M;
        int N, K, mode, bn, nst, split, persist;
        float ms;
    };
    std::vector<GemmTune> gemm_tune;
    // and the isosurface emit kernel's (element, isovalue) units per work-counter atomic, per
    // (order, elements, isovalues)
    struct EmitTune {
        int N, niso;
        int64_t E;
        int units;
        float ms;
    };
    std::vector<EmitTune> emit_tune;
    // and the launch width of persistent kernels (CTAs per SM, so elements per CTA) and the
    // render passes' grids, per (kernel, order, size); kind names the kernel (see LaunchTune)
    struct WidthTune {
        int kind, N;
        int64_t size;
        int width;
        float ms;
    };
    std::vector<WidthTune> width_tune;
    // device bytes the library holds for this context (scratch arenas, tables, meshes,
    // autoencoders) and their high-water mark
    int64_t mem_now = 0, mem_peak = 0;
    void mem_add(int64_t b)
    {
        mem_now += b;
        if (mem_now > mem_peak) mem_peak = mem_now;
    }
    // kernel trace: an event pair around every launch while tracing is on (not while the
    // stream is being captured); collected per kernel name by sem_trace_collect
    bool trace_on = false;
    struct TraceRec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<TraceRec> trace;
    std::vector<cudaEvent_t> trace_pool;
    struct TraceSum {
        const char *name;
        double ms;
        int64_t launches;
    };
    std::vector<TraceSum> trace_sum;
};

// Records ctx's trace events around the launch in its scope (see SEM_TRACED).
struct TraceScope {
    sem_ctx *ctx;
    int idx = -1;
    TraceScope(sem_ctx *c, const char *name);
    ~TraceScope();
};
#define SEM_TRACED(ctx, name, ...) \
    do {                           \
        TraceScope sem_ts_(ctx, name); \
        __VA_ARGS__;               \
    } while (0)

struct sem_mesh {
    int N = 0;
    int64_t E = 0;
    int device = 0;
    sem_ctx *owner = nullptr;  // the context whose memory count holds this mesh's bytes
    int64_t bytes = 0;
    float4 *lo = nullptr;   // element box lower corner (x0, y0, z0, 0)
    float4 *hi = nullptr;   // element box upper corner (x1, y1, z1, 0)
    float4 *g = nullptr;    // 2/(x1-x0), 2/(y1-y0), 2/(z1-z0), 0
    // general (curved) meshes: some element is not an axis-aligned affine box.  Then per node
    // the inverse Jacobian d r_d / d x_j (9 planes of E (N+1)^3 floats, plane 3 d + j) and the
    // node coordinates (3 planes); lo/hi hold each element's bounding box and g is zero.
    bool curved = false;
    float *geo = nullptr;
    float *xyzn = nullptr;
};


// set ctx->err and return st
sem_status sem_fail(sem_ctx *ctx, sem_status st, const char *fmt, ...);
// check a CUDA call; on failure records it and returns SEM_ERR_CUDA
sem_status sem_cuda(sem_ctx *ctx, cudaError_t e, const char *what);
// ensure scratch arena `slot` has at least `bytes`
sem_status sem_scratch(sem_ctx *ctx, int slot, size_t bytes, void **out);
// as sem_scratch, but refuses to grow the arena while ctx->stream is being captured into a graph
sem_status sem_scratch_nogrow_in_capture(sem_ctx *ctx, int slot, size_t bytes, void **out);

#define SEM_TRY(expr)                           \
    do {                                        \
        sem_status _st = (expr);                \
        if (_st != SEM_OK) return _st;          \
    } while (0)

#define SEM_CU(ctx, expr) SEM_TRY(sem_cuda((ctx), (expr), #expr))

// Per-(kernel, device) launch set-up.  The max-dynamic-shared-memory attribute and the resident
// blocks per SM belong to a kernel on one device, so they are set and computed once per device
// (the context's device, current when this runs) and cached in the kernel's own table.  Two
// host threads racing on a first call both set the same attribute and store the same value.
#define SEM_MAX_DEVICES 64
struct KernelSetup {
    std::atomic<int> per_sm[SEM_MAX_DEVICES];
};
template <class K>
inline sem_status kernel_setup(sem_ctx *ctx, KernelSetup &ks, K kern, int threads, size_t dyn, int *per_sm = nullptr)
{
    const int d = ctx->device;
    if (d < 0 || d >= SEM_MAX_DEVICES)
        return sem_fail(ctx, SEM_ERR_UNSUPPORTED, "device index %d: at most %d devices", d, SEM_MAX_DEVICES);
    int v = ks.per_sm[d].load(std::memory_order_acquire);
    if (!v) {
        SEM_CU(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        int nb = 1;
        if (threads > 0) {
            SEM_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, dyn));
            if (nb < 1) nb = 1;
        }
        ks.per_sm[d].store(nb, std::memory_order_release);
        v = nb;
    }
    if (per_sm) *per_sm = v;
    return SEM_OK;
}

// Launch-width autotuner of persistent kernels whose output does not depend on the width:
// the first call of a given (kind, N, size) with tuning on and the stream not being captured runs
// `launch(w)` for every candidate width (once untimed, then three times, each timed with CUDA
// events; a candidate's time is its fastest run), keeps the fastest and reuses it; otherwise
// `dflt`.  The last candidate's output is the call's output.
enum { TUNE_Q8 = 1, TUNE_Q8_COUNT = 2, TUNE_QGRAD = 3, TUNE_QGRAD_DERIV = 4, TUNE_RENDER = 5 };
template <class Launch>
inline sem_status width_tuned(sem_ctx *ctx, int kind, int N, int64_t size, const int *cand, int ncand, int dflt,
                              Launch launch)
{
    for (const auto &t : ctx->width_tune)
        if (t.kind == kind && t.N == N && t.size == size) return launch(t.width);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (!ctx->autotune || cs != cudaStreamCaptureStatusNone || ctx->trace_on || ncand < 2) return launch(dflt);
    cudaEvent_t e0, e1;
    SEM_CU(ctx, cudaEventCreate(&e0));
    SEM_CU(ctx, cudaEventCreate(&e1));
    int best = dflt;
    float best_ms = 1e30f;
    sem_status st = SEM_OK;
    for (int c = 0; c < ncand && st == SEM_OK; ++c) {
        st = launch(cand[c]);  // warm-up
        for (int rep = 0; rep < 3 && st == SEM_OK; ++rep) {
            st = sem_cuda(ctx, cudaEventRecord(e0, ctx->stream), "event");
            if (st == SEM_OK) st = launch(cand[c]);
            if (st == SEM_OK) st = sem_cuda(ctx, cudaEventRecord(e1, ctx->stream), "event");
            float ms = 0.f;
            if (st == SEM_OK) st = sem_cuda(ctx, cudaEventSynchronize(e1), "event");
            if (st == SEM_OK) st = sem_cuda(ctx, cudaEventElapsedTime(&ms, e0, e1), "event");
            if (st == SEM_OK && ms < best_ms) {
                best_ms = ms;
                best = cand[c];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SEM_TRY(st);
    ctx->width_tune.push_back({kind, N, size, best, best_ms});
    return SEM_OK;
}

static inline bool sem_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ------------------------------------------------------------------------------------------
// Per-translation-unit table uploads (constant memory lives in the unit that uses it)

// GLL derivative matrices (FP32) for N = 1..SEM_MAX_ORDER and node fractions (xi+1)/2
sem_status qcrit_upload_tables(sem_ctx *ctx, const float *D_all, const float *s_all);
sem_status iso_upload_tables(sem_ctx *ctx, const float *s_all, const int32_t *ntri, const int8_t *edges);

// launchers (argument checking happens in sem_api.cu)
sem_status qcrit_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                        float *Q);
// Q (N = 7 box meshes) and, in the same kernel, the per-element triangle counts cnt[q E + e] of
// Q's isosurfaces at isos[0..niso-1]
sem_status qcrit_count_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                              float *Q, int niso, const float *isos, int32_t *cnt);
sem_status qcrit_tc_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q,
                           sem_prec prec, const double *D64);
sem_status deriv_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, float *dx, float *dy, float *dz);
sem_status qcrit_batch_launch(sem_ctx *ctx, int n, const sem_mesh *const *m, const float *const *u,
                              const float *const *v, const float *const *w, float *const *Q);
sem_status iso_run(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris, int32_t *tri_elem,
                   int64_t cap, int64_t *ntri_out, uint8_t *cases);
sem_status iso_run_multi(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso, float *tris,
                         int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases);
sem_status iso_run_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso,
                               float *tris, int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases,
                               bool append = false);
// Q, its isosurfaces and those of nf further fields, appended behind Q's; the further fields'
// passes run on ctx->aux (see sem_qcriterion_isosurface_fields_async).  With `draw`, each
// group's segments are drawn into the frame begun by render_frame_begin right after its emit,
// on the stream that emitted them.
sem_status iso_run_q_fields_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                                  float *Q, const float *q_isos, int q_niso, int nf, const float *const *fields,
                                  const float *f_isos, const int *f_niso, float *tris, int32_t *tri_elem,
                                  int64_t cap, int64_t *counts_dev, bool draw = false);
sem_status iso_run_q_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                                 float *Q, const float *isos, int niso, float *tris, int32_t *tri_elem, int64_t cap,
                                 int64_t *counts_dev);
sem_status iso_run_noalloc(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                           int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases);
sem_status iso_noalloc_prepare(sem_ctx *ctx);
sem_status render_run(sem_ctx *ctx, const float *tris, int64_t ntri, const int64_t *seg_ntri, int nseg,
                      const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth,
                      const int64_t *seg_start_dev = nullptr, unsigned long long seg_mask = ~0ull);
// A frame drawn in parts (sem_frame_async): begun on ctx->stream (segment starts on the device,
// ntri_max the buffer's capacity), segments [seg_lo, seg_hi) drawn as part `part` (0..7, each
// part once per frame) on ctx->stream (whichever stream that is at the time), ended -- large triangles, resolve into rgba/depth -- on ctx->stream.
sem_status render_frame_begin(sem_ctx *ctx, int64_t ntri_max, const int64_t *seg_start_dev, int nseg,
                              const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth);
sem_status render_frame_draw(sem_ctx *ctx, const float *tris, int seg_lo, int seg_hi, int part);
sem_status render_frame_end(sem_ctx *ctx, const float *tris);
void render_frame_free(sem_ctx *ctx);
// true when the render's launch widths for W x H are chosen, or will not be timed
bool render_width_settled(sem_ctx *ctx, int W, int H);
sem_status measures_run(sem_ctx *ctx, const float *tris, int64_t ntri, double *out_host);
sem_status fieldmax_run(sem_ctx *ctx, const float *f, int64_t n, float *out_host);

// exclusive scan of n int32 counts into n+1 int64 offsets (out[n] = total).  `tmp` must hold
// scan_tmp_bytes(n) bytes.  Stream-ordered on ctx->stream.
size_t scan_tmp_bytes(int64_t n);
sem_status scan_i32_i64(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp);
// The same scan that also lists the entries with a positive count: live[0 .. *nlive) their
// indices in increasing order (live holds up to n entries).  `tmp` must hold
// scan_live_tmp_bytes(n) bytes.
size_t scan_live_tmp_bytes(int64_t n);
sem_status scan_i32_i64_live(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp, int64_t *live,
                             unsigned long long *nlive);
// makes the runtime load the scan kernels (lazy module loading), see iso_noalloc_prepare
sem_status scan_load_kernels(sem_ctx *ctx);

// ------------------------------------------------------------------------------------------
// Device helpers: mbarrier + bulk async copy (TMA engine, non-tensor form)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking test of a phase (for threads that poll several barriers)
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; returns false (and flags `err`) if the phase did not complete within `limit`
// polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  long long limit = SEM_WAIT_LIMIT)
{
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, 1 << SEM_ERR_TIMEOUT);
    return false;
}

// Orders this thread's earlier generic-proxy accesses of shared memory before later async-proxy
// ones (a bulk copy that overwrites what threads wrote there; the copy's issue must follow a
// barrier after the fence)
__device__ __forceinline__ void fence_proxy_async_cta() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// global -> shared bulk copy completing on `bar` (bytes: multiple of 16, both addresses 16B aligned)
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
