// sem_render.cu -- z-buffer rasteriser into a headless RGBA8 + depth image.
//
// Conventions (same statement as the header): pixel centres (x+.5, y+.5), edge functions with
// the top-left fill rule on the triangle made clockwise on screen (y down), zero-area and
// near/far-crossing triangles dropped, depth interpolated in screen space, smallest
// (depth, triangle index) wins, flat headlight shading c = rgb (0.15 + 0.85 |n.l|).
//
// Depth resolve: one 64-bit key per pixel, (depth bits << 32) | triangle index, combined with
// atomicMin -- the minimum is order-independent, so the image is deterministic.  The key
// buffer (8 B/pixel: 16.6 MB at 1920x1080) stays resident in the 129 MB L2.
//
// Passes (no host synchronisation):
//   k_raster_small   one thread per triangle (staged through shared memory): project,
//                    normalise winding, take the exact range of pixel centres its bounding box
//                    contains (sub-pixel triangles that contain none are done); for boxes of at
//                    most SMALL_PX centres, the warp spreads all its triangles' centre tests
//                    evenly over its lanes and atomicMins the keys.  Larger triangles are
//                    appended to a list.  One 256-triangle tile per block.
//   k_raster_masked  the same per tile, for a frame with a draw mask: a persistent grid over the
//                    drawn segments' tiles only.
//   k_raster_range   the same per tile, for a frame drawn in parts (sem_frame_async): a
//                    persistent grid over the tiles of one part's device range of segments,
//                    launched on the stream that produced that part's triangles.
//   k_raster_large   one warp per listed triangle, its lanes stepping 32 candidates at a time
//                    on the triangle's planes.
//   k_resolve        grid-stride over groups of four pixels: read the key, reset it for the next
//                    frame, look up the winner's colour (computed by the raster pass).
//
// Why not per-tile shared-memory z-buffers: the isosurface frames consist of millions of
// triangles a few pixels or less in size, and binning them into tile lists costs two extra
// passes over the triangle data plus contended per-tile counters (measured: binning and the
// tile raster took 88% of the frame).  Direct L2 atomics do it in one pass.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sem_internal.cuh"

#define SMALL_PX 32        // boxes with at most this many pixel centres: the warp's candidate list
#define LARGE_THREADS 256
#define RENDER_MAX_SEG 64  // segments of sem_render_segments_async (16 for sem_render, sem_render_async)

struct RenderParams {
    float eye[3], s[3], u[3], f[3];
    float ax, ay;        // projection scales
    float znear, zfar;   // clip range on z_view
    float za, zb;        // depth: ortho (zv - znear)*za ; perspective zb*(1 - znear/zv)
    int ortho;
    int W, H;
    float hw, hh;        // W / 2, H / 2 (viewport: sx = hw (xn + 1), sy = hh (1 - yn))
    float wmax, hmax;    // W - 1, H - 1
    int nseg;
    int seg_end[RENDER_MAX_SEG];
    float rgb[RENDER_MAX_SEG][3];
    const int64_t *seg_dev;  // device segment starts [nseg + 1] (asynchronous render), or null
    unsigned long long seg_mask;  // bit s set: segment s is drawn (all ones: every segment)
};

// Screen position of one vertex; the NDC depth is finished in setup_tri only for triangles that
// cover a pixel centre, from zw: the view depth (orthographic) or its reciprocal (perspective:
// one __frcp_rn, correctly rounded, per vertex, shared by the position and the depth).
__device__ __forceinline__ bool project(const RenderParams &P, const float *p, float &sx, float &sy, float &zw)
{
    const float dx = p[0] - P.eye[0], dy = p[1] - P.eye[1], dz = p[2] - P.eye[2];
    const float xv = P.s[0] * dx + P.s[1] * dy + P.s[2] * dz;
    const float yv = P.u[0] * dx + P.u[1] * dy + P.u[2] * dz;
    const float zv = P.f[0] * dx + P.f[1] * dy + P.f[2] * dz;
    if (!(zv > P.znear && zv < P.zfar)) return false;
    float xn, yn;
    if (P.ortho) {
        xn = xv * P.ax;
        yn = yv * P.ay;
        zw = zv;
    } else {
        const float rz = __frcp_rn(zv);
        xn = xv * rz * P.ax;
        yn = yv * rz * P.ay;
        zw = rz;
    }
    sx = fmaf(xn, P.hw, P.hw);
    sy = fmaf(-yn, P.hh, P.hh);
    return true;
}

__device__ __forceinline__ float ndc_depth(const RenderParams &P, float zw)
{
    return P.ortho ? (zw - P.znear) * P.za : P.zb * (1.f - P.znear * zw);
}

// Screen-space setup of one triangle; false if it is dropped or contains no pixel centre.
struct Setup {
    float x[3], y[3], z[3];
    float inv_area;
    int px0, px1, py0, py1;
};

__device__ __forceinline__ bool setup_tri(const RenderParams &P, const float *__restrict__ p, Setup &S)
{
    float zv0, zv1, zv2;
    if (!(project(P, p, S.x[0], S.y[0], zv0) && project(P, p + 3, S.x[1], S.y[1], zv1) &&
          project(P, p + 6, S.x[2], S.y[2], zv2)))
        return false;
    // pixel centres c = p + 0.5 inside the box: ceil(min - .5) <= p <= floor(max - .5); most
    // small triangles contain none and stop here
    const float mnx = fminf(S.x[0], fminf(S.x[1], S.x[2])), mxx = fmaxf(S.x[0], fmaxf(S.x[1], S.x[2]));
    const float mny = fminf(S.y[0], fminf(S.y[1], S.y[2])), mxy = fmaxf(S.y[0], fmaxf(S.y[1], S.y[2]));
    const float fx0 = fmaxf(0.f, ceilf(mnx - 0.5f)), fx1 = fminf(P.wmax, floorf(mxx - 0.5f));
    const float fy0 = fmaxf(0.f, ceilf(mny - 0.5f)), fy1 = fminf(P.hmax, floorf(mxy - 0.5f));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
    float area = (S.x[1] - S.x[0]) * (S.y[2] - S.y[0]) - (S.x[2] - S.x[0]) * (S.y[1] - S.y[0]);
    if (!(area != 0.f) || isnan(area)) return false;
    S.z[0] = ndc_depth(P, zv0);
    S.z[1] = ndc_depth(P, zv1);
    S.z[2] = ndc_depth(P, zv2);
    if (area < 0.f) {
        float tx = S.x[1], ty = S.y[1], tz = S.z[1];
        S.x[1] = S.x[2]; S.y[1] = S.y[2]; S.z[1] = S.z[2];
        S.x[2] = tx; S.y[2] = ty; S.z[2] = tz;
        area = -area;
    }
    S.px0 = (int)fx0;
    S.px1 = (int)fx1;
    S.py0 = (int)fy0;
    S.py1 = (int)fy1;
    S.inv_area = 1.f / area;
    return true;
}

// Compact per-triangle setup kept in shared memory for the warp's pixel work: the three edge
// functions and the depth as planes over the triangle's box, e(kx, ky) = e(0, 0) + A kx + B ky
// for candidate (px0 + kx, py0 + ky), so a test is eight FMAs.  The values at the box's first
// pixel centre are the edge functions (x_i+1 - x_i)(cy - y_i) - (y_i+1 - y_i)(cx - x_i) of the
// edges v0 v1, v1 v2, v2 v0; the increments are the edges' coordinate differences.  Per
// triangle, in four arrays (a lane's stores are contiguous with its neighbours'):
//   a: e0 e1 e2 z at (px0 + .5, py0 + .5)   b: de/dx (3), dz/dx   c: de/dy (3), dz/dy
//   d: pixel index py0 W + px0,  ceil(1024 / nx),  nx,  top-left flags (one per byte)
// Box row of candidate k (0 <= k < nx ny <= 32): ky = (k ceil(1024/nx)) >> 10 is floor(k/nx)
// exactly, since k (ceil(1024/nx) - 1024/nx) / 1024 < k / 1024 < 1/nx for nx < 32, and the
// multiplier is exact for nx = 32.
//
// Coverage test on the float bits: for a float e that is neither -0 nor NaN,
// "e > 0, or e == 0 on a top-left edge" is exactly int_bits(e) + tl > 0 (positive floats have
// positive integer bits, +0 has 0, negative floats negative ones).  The box-origin values are
// stored with -0 turned into +0 (x + 0 = +0 for x = -0), and an FMA chain of such a value with
// non-negative candidate offsets rounds an exact zero to +0, never -0.  Triangles whose planes
// could overflow within their box (|e| + span (|A| + |B|) not finite, span 32 for the small
// boxes and the longer side for the others) are not drawn, so no test sees an infinity or NaN.
struct SmallRecs {
    float4 a[256], b[256], c[256];
    int4 d[256];
};

// The planes of triangle S over its box (see above); false if they could overflow within
// `span` pixels of the box origin.  tl: the top-left flags, one per byte.
__device__ __forceinline__ bool make_planes(const Setup &S, float span, float4 &pa, float4 &pb, float4 &pc, int &tl)
{
    const float cx = (float)S.px0 + 0.5f, cy = (float)S.py0 + 0.5f;
    const float e0 = (S.x[1] - S.x[0]) * (cy - S.y[0]) - (S.y[1] - S.y[0]) * (cx - S.x[0]) + 0.f;
    const float e1 = (S.x[2] - S.x[1]) * (cy - S.y[1]) - (S.y[2] - S.y[1]) * (cx - S.x[1]) + 0.f;
    const float e2 = (S.x[0] - S.x[2]) * (cy - S.y[2]) - (S.y[0] - S.y[2]) * (cx - S.x[2]) + 0.f;
    const float A0 = S.y[0] - S.y[1], A1 = S.y[1] - S.y[2], A2 = S.y[2] - S.y[0];
    const float B0 = S.x[1] - S.x[0], B1 = S.x[2] - S.x[1], B2 = S.x[0] - S.x[2];
    const float z = (e1 * S.z[0] + e2 * S.z[1] + e0 * S.z[2]) * S.inv_area;
    const float dzdx = (A1 * S.z[0] + A2 * S.z[1] + A0 * S.z[2]) * S.inv_area;
    const float dzdy = (B1 * S.z[0] + B2 * S.z[1] + B0 * S.z[2]) * S.inv_area;
    const float reach = fabsf(e0) + fabsf(e1) + fabsf(e2) + fabsf(z) +
                        span * (fabsf(A0) + fabsf(A1) + fabsf(A2) + fabsf(B0) + fabsf(B1) + fabsf(B2) +
                                fabsf(dzdx) + fabsf(dzdy));
    if (!(reach <= 3.0e38f)) return false;
    // top-left: dy < 0, or dy == 0 and dx > 0, with dy = -A_i and dx = B_i of edge i (exact)
    tl = ((A0 > 0.f || (A0 == 0.f && B0 > 0.f)) ? 1 : 0) | ((A1 > 0.f || (A1 == 0.f && B1 > 0.f)) ? 0x100 : 0) |
         ((A2 > 0.f || (A2 == 0.f && B2 > 0.f)) ? 0x10000 : 0);
    pa = make_float4(e0, e1, e2, z);
    pb = make_float4(A0, A1, A2, dzdx);
    pc = make_float4(B0, B1, B2, dzdy);
    return true;
}

// Coverage of candidate (kx, ky) >= 0 of the box and its depth, from the planes; see above
// for why the integer test equals the top-left rule.
__device__ __forceinline__ bool plane_test(const float4 &a, const float4 &b, const float4 &c, int tl, float fx, float fy,
                                           float &z)
{
    const int v0 = __float_as_int(fmaf(c.x, fy, fmaf(b.x, fx, a.x))) + (int)__byte_perm(tl, 0, 0x4440);
    const int v1 = __float_as_int(fmaf(c.y, fy, fmaf(b.y, fx, a.y))) + (int)__byte_perm(tl, 0, 0x4441);
    const int v2 = __float_as_int(fmaf(c.z, fy, fmaf(b.z, fx, a.z))) + (int)__byte_perm(tl, 0, 0x4442);
    z = fminf(fmaxf(fmaf(c.w, fy, fmaf(b.w, fx, a.w)), 0.f), 1.f);
    return min(v0, min(v1, v2)) > 0;
}

__device__ __forceinline__ bool store_rec(SmallRecs &R, int i, const Setup &S, int W)
{
    float4 a, b, c;
    int tl;
    if (!make_planes(S, 32.f, a, b, c, tl)) return false;
    const int nx = S.px1 - S.px0 + 1;
    // ceil(1024 / nx): 1024/nx is an integer or at least 1/32 above one, far beyond the
    // approximate quotient's error
    const int mul = (int)(__fdividef(1024.f, (float)nx) - 0.00390625f) + 1;
    R.a[i] = a;
    R.b[i] = b;
    R.c[i] = c;
    R.d[i] = make_int4(S.py0 * W + S.px0, mul, nx, tl);
    return true;
}

// Flat headlight shade of triangle t (colour of its segment times 0.15 + 0.85 |n.l|, l the view
// direction), packed as RGBA8 with alpha 255.
__device__ __forceinline__ uint32_t shade_rgba(const RenderParams &P, const float *__restrict__ p, int sg)
{
    const float ax = p[3] - p[0], ay = p[4] - p[1], az = p[5] - p[2];
    const float bx = p[6] - p[0], by = p[7] - p[1], bz = p[8] - p[2];
    const float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
    const float n2 = nx * nx + ny * ny + nz * nz;
    const float shade = n2 > 0.f ? 0.15f + 0.85f * fabsf(nx * P.f[0] + ny * P.f[1] + nz * P.f[2]) * rsqrtf(n2) : 0.15f;
    uint32_t c = 0xff000000u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // floor(v 255 + .5) of v = clamp(rgb shade, 0, 1): a value in [.5, 255.5]
        const float v = __saturatef(P.rgb[sg][k] * shade);
        c |= __float2uint_rd(fmaf(v, 255.f, 0.5f)) << (8 * k);
    }
    return c;
}

// start of segment k (k <= nseg): device table (asynchronous render) or the parameter ends
__device__ __forceinline__ int64_t seg_start(const RenderParams &P, int k)
{
    if (P.seg_dev) return __ldg(P.seg_dev + k);
    return k == 0 ? 0 : (int64_t)P.seg_end[k - 1];
}


// Shared memory of one block's tile of up to 256 triangles.
struct RasterSmem {
    __align__(16) float tri[256 * 9];
    SmallRecs rec;
    uint8_t lane_of[8][32];
    int64_t seg[RENDER_MAX_SEG + 1];  // starts of the drawn segments seg_lo .. seg_hi (the last: an end)
    int any;                          // some triangle of the tile lies in a drawn segment
};

// segment of triangle t (relative to seg_lo) from the starts in shared memory: the last k < ns
// with seg[k] <= t
__device__ __forceinline__ int seg_index(const int64_t *seg, int ns, int64_t t)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One tile: triangles t0 .. t0 + nt - 1, all in segments seg_lo .. seg_hi - 1.  The block first
// reads the starts of those segments and the end of the last into shared memory (one load per
// segment, in parallel; only these, as a frame drawn in parts has other parts' starts written by
// other streams); with a draw mask, a tile whose triangles all lie in segments that are not
// drawn is done before its triangles are read.
// Then one thread per triangle for the setup (its 36 bytes staged through shared memory with
// coalesced loads, its segment by binary search); then each warp spreads the pixel-centre
// tests of its 32 triangles evenly over its lanes, so a lane never idles while a neighbour walks
// a bigger box; a pixel test finds its triangle from one warp OR of the list starts in its round
// and a rank -> lane table.  Block-uniform exits only; the caller synchronises the block before
// it reuses `sm`.
__device__ __forceinline__ void raster_tile(const float *__restrict__ tris, int t0, int nt_blk, int seg_lo,
                                            int seg_hi, const RenderParams &P, unsigned long long *__restrict__ keys,
                                            int32_t *__restrict__ large, int32_t *__restrict__ nlarge,
                                            uint32_t *__restrict__ colors, RasterSmem &sm, bool check_mask = true)
{
    const int ns = seg_hi - seg_lo;
    if ((int)threadIdx.x <= ns) sm.seg[threadIdx.x] = seg_start(P, seg_lo + threadIdx.x);
    if (check_mask && P.seg_mask != ~0ull) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int a = seg_lo + seg_index(sm.seg, ns, t0), b = seg_lo + seg_index(sm.seg, ns, t0 + nt_blk - 1);
            // segments a .. b (b - a < 64)
            const unsigned long long span = (b - a == 63) ? ~0ull : (((2ull << (b - a)) - 1ull) << a);
            sm.any = (P.seg_mask & span) != 0ull;
        }
        __syncthreads();
        if (!sm.any) return;
    }
    float *s_tri = sm.tri;
    const float *src = tris + (int64_t)t0 * 9;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        // 16-byte loads when the tile's 36-byte triangles start on a 16-byte boundary
        const int n4 = nt_blk * 9 / 4;
        for (int q = threadIdx.x; q < n4; q += 256)
            reinterpret_cast<float4 *>(s_tri)[q] = __ldcs(reinterpret_cast<const float4 *>(src) + q);
        for (int q = n4 * 4 + threadIdx.x; q < nt_blk * 9; q += 256) s_tri[q] = __ldcs(src + q);
    } else {
        for (int q = threadIdx.x; q < nt_blk * 9; q += 256) s_tri[q] = __ldcs(src + q);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int t = t0 + threadIdx.x;
    bool is_large = false;
    int npx = 0;
    const int sg = (int)threadIdx.x < nt_blk ? seg_lo + seg_index(sm.seg, ns, t) : 0;
    if ((int)threadIdx.x < nt_blk && ((P.seg_mask >> sg) & 1ull)) {
        Setup S;
        if (setup_tri(P, s_tri + threadIdx.x * 9, S)) {
            // only triangles that cover a pixel centre can win a pixel: their colour, once
            colors[t] = shade_rgba(P, s_tri + threadIdx.x * 9, sg);
            const int nx = S.px1 - S.px0 + 1, ny = S.py1 - S.py0 + 1;
            if (nx * ny <= SMALL_PX) {
                if (store_rec(sm.rec, threadIdx.x, S, P.W)) npx = nx * ny;
            } else {
                is_large = true;
            }
        }
    }
    // warp-aggregated append of the large triangles
    const unsigned m = __ballot_sync(0xffffffffu, is_large);
    if (m) {
        int base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(nlarge, __popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (is_large) large[base + __popc(m & ((1u << lane) - 1u))] = t;
    }
    // inclusive scan of the pixel counts over the warp
    int incl = npx;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int wbase = threadIdx.x & ~31;
    const int excl = incl - npx;
    // owners: the lanes with candidates, in lane order; their lists start at excl, increasing.
    // Owner rank -> lane in a 32-byte table.
    const unsigned owners = __ballot_sync(0xffffffffu, npx > 0);
    uint8_t *lane_of = sm.lane_of[threadIdx.x >> 5];
    if (npx > 0) lane_of[__popc(owners & ((1u << lane) - 1u))] = (uint8_t)lane;
    __syncwarp();
    // each round: lane `lane` takes candidate r + lane of the warp's list.  The owners whose
    // lists start in [r, r + 32) set one bit each (warp OR); the candidate's owner has rank
    // (starts before r) + (starts at or below it in the window) - 1.  Branch-free up to the
    // atomic: past the list's end the rank is the last owner's, and the candidate is switched
    // off in the coverage predicate.
    const int W = P.W;
    int before = 0;
    for (int r = 0; r < total; r += 32) {
        const int idx = r + lane;
        const unsigned starts =
            __reduce_or_sync(0xffffffffu, (npx > 0 && (unsigned)(excl - r) < 32u) ? 1u << (excl - r) : 0u);
        const int rank = before + __popc(starts & ((2u << lane) - 1u)) - 1;
        before += __popc(starts);
        const int L = lane_of[rank & 31];
        const int first = __shfl_sync(0xffffffffu, excl, L);
        const int i = wbase + L;
        const float4 a = sm.rec.a[i], b = sm.rec.b[i], c = sm.rec.c[i];
        const int4 d = sm.rec.d[i];
        const int k = idx - first;
        const int ky = (k * d.y) >> 10, kx = k - ky * d.z;
        float z;
        if (plane_test(a, b, c, d.w, (float)kx, (float)ky, z) && idx < total) {
            const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)(t0 + i);
            atomicMin(keys + (unsigned)(d.x + ky * W + kx), key);
        }
    }
}

// One tile of 256 triangles per block, triangles [0, ntri) (ntri clamped to the device start of
// segment seg_end -- the total for a whole frame -- when the segments come from the device).
__global__ void __launch_bounds__(256) k_raster_small(const float *__restrict__ tris, int ntri, int seg_end,
                                                      const __grid_constant__ RenderParams P,
                                                      unsigned long long *__restrict__ keys,
                                                      int32_t *__restrict__ large, int32_t *__restrict__ nlarge,
                                                      uint32_t *__restrict__ colors)
{
    __shared__ RasterSmem sm;
    if (P.seg_dev) ntri = (int)min((int64_t)ntri, P.seg_dev[seg_end]);
    const int t0 = blockIdx.x * 256;
    // blocks past the (device-clamped) triangle count have no work; the whole block leaves
    // before its first barrier
    if (t0 >= ntri) return;
    raster_tile(tris, t0, min(256, ntri - t0), 0, seg_end, P, keys, large, nlarge, colors, sm);
}

// The triangles of segments [seg_lo, seg_hi), their range read from the device segment starts
// and clamped to the buffer's ntri: a persistent grid whose blocks take the 256-triangle tiles
// of the whole buffer that meet the range from a counter (zeroed when the frame begins), so they
// finish within a tile of each other; the tiles stay on the buffer's 256-triangle grid (only the
// range's first tile can start unaligned) and are clipped to the range.  Used where a frame is
// drawn in parts, one part per stream, before one resolve.
__global__ void __launch_bounds__(256, 6) k_raster_range(const float *__restrict__ tris, int ntri, int seg_lo,
                                                         int seg_hi, const __grid_constant__ RenderParams P,
                                                         unsigned long long *__restrict__ keys,
                                                         int32_t *__restrict__ large, int32_t *__restrict__ nlarge,
                                                         uint32_t *__restrict__ colors, int *__restrict__ next_tile)
{
    __shared__ RasterSmem sm;
    __shared__ int s_k[2];  // the current tile's counter value and the next one's
    // clamped to the buffer's capacity, as k_raster_small clamps the device total
    const int64_t hi = min(seg_start(P, seg_hi), (int64_t)ntri), lo = min(seg_start(P, seg_lo), hi);
    if (threadIdx.x == 0) s_k[0] = atomicAdd(next_tile, 1);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const int64_t tile = lo / 256 + s_k[cur];
        if (tile * 256 >= hi) break;  // block-uniform
        // the next tile's counter value, fetched while this one is drawn (read after the barrier
        // at the end of this iteration)
        if (threadIdx.x == 0) s_k[cur ^ 1] = atomicAdd(next_tile, 1);
        const int64_t a = max(tile * 256, lo), b = min(tile * 256 + 256, hi);
        raster_tile(tris, (int)a, (int)(b - a), seg_lo, seg_hi, P, keys, large, nlarge, colors, sm);
        __syncthreads();  // the tile's shared memory is free for the next
    }
}

// The drawn segments of a frame with a draw mask: a persistent grid whose blocks take the tiles
// of the drawn segments only, from a counter (zeroed when the frame begins).  Each block lists
// the drawn segments' 256-triangle tiles (the buffer's tile grid, clipped to the segment) with a
// prefix sum over at most 64 segments in shared memory, and maps each tile it takes to its
// segment by binary search; a tile shared by two drawn segments is two work items.  No block
// reads the triangles of a segment that is not drawn.
struct MaskedSmem {
    int64_t start[RENDER_MAX_SEG + 1];  // the frame's segment starts (clamped to the buffer)
    int64_t first[RENDER_MAX_SEG + 1];  // work items before the k-th drawn segment
    int seg[RENDER_MAX_SEG];            // the drawn segments, in order
    int ndrawn;
    int k[2];                           // the current work item's counter value and the next one's
};

__global__ void __launch_bounds__(256, 6) k_raster_masked(const float *__restrict__ tris, int ntri,
                                                          const __grid_constant__ RenderParams P,
                                                          unsigned long long *__restrict__ keys,
                                                          int32_t *__restrict__ large, int32_t *__restrict__ nlarge,
                                                          uint32_t *__restrict__ colors, int *__restrict__ next_item)
{
    __shared__ RasterSmem sm;
    __shared__ MaskedSmem ms;
    if ((int)threadIdx.x <= P.nseg) ms.start[threadIdx.x] = min(seg_start(P, threadIdx.x), (int64_t)ntri);
    if (threadIdx.x == 0) ms.k[0] = atomicAdd(next_item, 1);
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp 0: the drawn segments with their tile counts, a prefix sum over them
        const int lane = threadIdx.x;
        int64_t before = 0;
        int nd = 0;
        for (int s0 = 0; s0 < P.nseg; s0 += 32) {
            const int sg = s0 + lane;
            int64_t tiles = 0;
            const bool drawn = sg < P.nseg && ((P.seg_mask >> sg) & 1ull);
            if (drawn) {
                const int64_t a = ms.start[sg], b = ms.start[sg + 1];
                tiles = b > a ? (b + 255) / 256 - a / 256 : 0;
            }
            const bool live = drawn && tiles > 0;
            const unsigned bal = __ballot_sync(0xffffffffu, live);
            int64_t incl = tiles;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (live) {
                const int r = nd + __popc(bal & ((1u << lane) - 1u));
                ms.seg[r] = sg;
                ms.first[r] = before + incl - tiles;
            }
            nd += __popc(bal);
            before += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            ms.ndrawn = nd;
            ms.first[nd] = before;
        }
    }
    __syncthreads();
    const int nd = ms.ndrawn;
    for (int cur = 0;; cur ^= 1) {
        const int64_t item = ms.k[cur];
        if (item >= ms.first[nd]) break;  // block-uniform
        if (threadIdx.x == 0) ms.k[cur ^ 1] = atomicAdd(next_item, 1);
        // the drawn segment holding work item `item`: the last r with first[r] <= item
        int lo = 0, hi = nd - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ms.first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int sg = ms.seg[lo];
        const int64_t a0 = ms.start[sg], b0 = ms.start[sg + 1];
        const int64_t tile = a0 / 256 + (item - ms.first[lo]);
        const int64_t a = max(tile * 256, a0), b = min(tile * 256 + 256, b0);
        raster_tile(tris, (int)a, (int)(b - a), sg, sg + 1, P, keys, large, nlarge, colors, sm, false);
        __syncthreads();  // the tile's shared memory is free for the next
    }
}

// Triangles with more than SMALL_PX candidate pixels: one warp per triangle, lane l taking
// candidates l, l + 32, ... of the box in row order (one division per triangle, then each
// step of 32 candidates is q rows and r columns), tested on the triangle's planes.
__global__ void __launch_bounds__(LARGE_THREADS) k_raster_large(const float *__restrict__ tris,
                                                                const int32_t *__restrict__ large,
                                                                const int32_t *__restrict__ nlarge,
                                                                const __grid_constant__ RenderParams P,
                                                                unsigned long long *__restrict__ keys)
{
    const int n = *nlarge;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (LARGE_THREADS / 32);
    for (int q = blockIdx.x * (LARGE_THREADS / 32) + (threadIdx.x >> 5); q < n; q += warps) {
        const int t = large[q];
        Setup S;
        if (!setup_tri(P, tris + (int64_t)t * 9, S)) continue;
        const int nx = S.px1 - S.px0 + 1, ny = S.py1 - S.py0 + 1;
        float4 a, b, c;
        int tl;
        if (!make_planes(S, (float)max(nx, ny), a, b, c, tl)) continue;
        const int dq = 32 / nx, dr = 32 - dq * nx;
        int ky = lane / nx, kx = lane - ky * nx;
        while (ky < ny) {
            float z;
            if (plane_test(a, b, c, tl, (float)kx, (float)ky, z)) {
                const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)t;
                atomicMin(keys + (unsigned)((S.py0 + ky) * P.W + S.px0 + kx), key);
            }
            kx += dr;
            ky += dq;
            if (kx >= nx) {
                kx -= nx;
                ++ky;
            }
        }
    }
}

// Per pixel: the winning key's depth and its triangle's colour (computed by the raster pass);
// resets the key for the next frame.  Grid-stride over groups of four pixels (16-byte key,
// colour and depth accesses); the last npx % 4 pixels go to the first threads.
__device__ __forceinline__ void resolve_one(unsigned long long key, const uint32_t *__restrict__ colors, uint32_t &c,
                                            float &d)
{
    if (key == ~0ull) {
        c = 0u;
        d = 1.f;
    } else {
        c = colors[key & 0xffffffffu];
        d = __uint_as_float((unsigned)(key >> 32));
    }
}

__global__ void __launch_bounds__(256) k_resolve(const uint32_t *__restrict__ colors, int64_t npx,
                                                 unsigned long long *__restrict__ keys, uint32_t *__restrict__ rgba,
                                                 float *__restrict__ depth)
{
    const int64_t n4 = npx >> 2, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(keys);
    const ulonglong2 empty = make_ulonglong2(~0ull, ~0ull);
    for (int64_t q = tid; q < n4; q += stride) {
        const ulonglong2 a = k2[2 * q], b = k2[2 * q + 1];
        // ready for the next frame: only keys some triangle wrote need resetting (most pixels of
        // an isosurface frame stay background and already hold "empty")
        if ((a.x & a.y) != ~0ull) k2[2 * q] = empty;
        if ((b.x & b.y) != ~0ull) k2[2 * q + 1] = empty;
        uint4 c;
        float4 d;
        resolve_one(a.x, colors, c.x, d.x);
        resolve_one(a.y, colors, c.y, d.y);
        resolve_one(b.x, colors, c.z, d.z);
        resolve_one(b.y, colors, c.w, d.w);
        __stcs(reinterpret_cast<uint4 *>(rgba) + q, c);
        if (depth) __stcs(reinterpret_cast<float4 *>(depth) + q, d);
    }
    const int64_t pix = 4 * n4 + tid;
    if (pix < npx) {
        const unsigned long long key = keys[pix];
        keys[pix] = ~0ull;
        uint32_t c;
        float d;
        resolve_one(key, colors, c, d);
        rgba[pix] = c;
        if (depth) depth[pix] = d;
    }
}

static const float kPalette[16][3] = {
    {0.90f, 0.35f, 0.25f}, {0.25f, 0.60f, 0.90f}, {0.35f, 0.85f, 0.40f}, {0.95f, 0.80f, 0.25f},
    {0.70f, 0.40f, 0.85f}, {0.30f, 0.85f, 0.85f}, {0.95f, 0.55f, 0.75f}, {0.60f, 0.60f, 0.60f},
    {0.80f, 0.50f, 0.20f}, {0.20f, 0.40f, 0.70f}, {0.50f, 0.70f, 0.20f}, {0.90f, 0.90f, 0.90f},
    {0.55f, 0.25f, 0.45f}, {0.20f, 0.65f, 0.55f}, {0.85f, 0.30f, 0.55f}, {0.40f, 0.40f, 0.80f}};

static void unit3(double *a)
{
    const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= n;
    a[1] /= n;
    a[2] /= n;
}

// A frame's parameters and buffers: the key buffer (kept all "empty" between frames), the
// large-triangle counter and list, the per-triangle colours.
#define RENDER_MAX_PARTS 8  // parts of a frame drawn in parts, each with its tile counter
struct RenderFrame {
    RenderParams P;
    unsigned long long *keys = nullptr;
    int32_t *nlarge = nullptr, *large = nullptr;
    int *next_tile = nullptr;  // [RENDER_MAX_PARTS] tile counters of the parts
    uint32_t *colors = nullptr;
    int ntri = 0;
    int64_t npx = 0;
    uint8_t *rgba = nullptr;
    float *depth = nullptr;
};

// Projection, segment table and buffers of one frame (no launch but the one-time reset of a new
// key buffer, on ctx->stream).
static sem_status render_setup(sem_ctx *ctx, RenderFrame &F, int64_t ntri64, const int64_t *seg_ntri, int nseg,
                               const float *seg_rgb, const sem_camera *cam, int W, int H,
                               const int64_t *seg_start_dev, unsigned long long seg_mask)
{
    if (nseg < 1 || nseg > RENDER_MAX_SEG) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: nseg=%d", nseg);
    RenderParams &P = F.P;
    memset(&P, 0, sizeof P);
    double f[3], s[3], u[3], up[3];
    for (int k = 0; k < 3; ++k) {
        f[k] = (double)cam->center[k] - (double)cam->eye[k];
        up[k] = cam->up[k];
    }
    if (!(f[0] * f[0] + f[1] * f[1] + f[2] * f[2] > 0.0))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_render: eye and center coincide");
    unit3(f);
    s[0] = f[1] * up[2] - f[2] * up[1];
    s[1] = f[2] * up[0] - f[0] * up[2];
    s[2] = f[0] * up[1] - f[1] * up[0];
    if (!(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] > 0.0))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_render: up is parallel to the view direction");
    unit3(s);
    u[0] = s[1] * f[2] - s[2] * f[1];
    u[1] = s[2] * f[0] - s[0] * f[2];
    u[2] = s[0] * f[1] - s[1] * f[0];
    for (int k = 0; k < 3; ++k) {
        P.eye[k] = cam->eye[k];
        P.f[k] = (float)f[k];
        P.s[k] = (float)s[k];
        P.u[k] = (float)u[k];
    }
    const double aspect = (double)W / (double)H;
    P.ortho = cam->ortho != 0;
    if (P.ortho) {
        P.ax = (float)(1.0 / ((double)cam->half_h * aspect));
        P.ay = (float)(1.0 / (double)cam->half_h);
        P.za = (float)(1.0 / ((double)cam->zfar - (double)cam->znear));
    } else {
        const double th = tan(0.5 * (double)cam->fovy_deg * M_PI / 180.0);
        P.ax = (float)(1.0 / (th * aspect));
        P.ay = (float)(1.0 / th);
        P.zb = (float)((double)cam->zfar / ((double)cam->zfar - (double)cam->znear));
    }
    P.znear = cam->znear;
    P.zfar = cam->zfar;
    P.W = W;
    P.H = H;
    P.hw = 0.5f * (float)W;
    P.hh = 0.5f * (float)H;
    P.wmax = (float)(W - 1);
    P.hmax = (float)(H - 1);
    P.nseg = nseg;
    P.seg_dev = seg_start_dev;
    P.seg_mask = nseg == 64 ? seg_mask : (seg_mask | ~((1ull << nseg) - 1ull));
    int64_t acc = 0;
    for (int k = 0; k < nseg; ++k) {
        acc += seg_ntri[k];
        P.seg_end[k] = (int)acc;
        for (int c = 0; c < 3; ++c) P.rgb[k][c] = seg_rgb ? seg_rgb[3 * k + c] : kPalette[k % 16][c];
    }
    const int ntri = (int)ntri64;
    const int64_t npx = (int64_t)W * H;
    // scratch: key buffer (kept all-ones between frames) in its own arena; the large-triangle
    // counter and list in another
    const size_t b_keys = sizeof(unsigned long long) * (size_t)npx;
    void *kscr = nullptr, *lscr = nullptr;
    void *const prev = ctx->scratch[SCR_RENDER];
    const size_t prev_bytes = ctx->scratch_bytes[SCR_RENDER];
    SEM_TRY(sem_scratch_nogrow_in_capture(ctx, SCR_RENDER, b_keys, &kscr));
    if (kscr != prev || ctx->scratch_bytes[SCR_RENDER] != prev_bytes || ctx->render_keys_dirty) {
        // a new arena holds no valid keys yet: set every key to "empty" once
        SEM_CU(ctx, cudaMemsetAsync(kscr, 0xff, ctx->scratch_bytes[SCR_RENDER], ctx->stream));
        ctx->render_keys_dirty = false;
    }
    // large-triangle counter, list (int32 per triangle) and per-triangle colours (RGBA8)
    const size_t nt1 = (size_t)(ntri > 0 ? ntri : 1);
    const size_t list_bytes = ((sizeof(int32_t) * nt1 + 255) / 256) * 256;
    SEM_TRY(sem_scratch_nogrow_in_capture(ctx, SCR_TRI, 256 + list_bytes + sizeof(uint32_t) * nt1, &lscr));
    F.keys = reinterpret_cast<unsigned long long *>(kscr);
    F.nlarge = reinterpret_cast<int32_t *>(lscr);
    F.next_tile = reinterpret_cast<int *>(lscr) + 1;
    F.large = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(lscr) + 256);
    F.colors = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(lscr) + 256 + list_bytes);
    F.ntri = ntri;
    F.npx = npx;
    return SEM_OK;
}

// the widths of the persistent large-triangle pass and of the resolve pass (in CTAs per SM), one
// pair per candidate of the context's autotuner, chosen per frame size on the first frame
static const int kLarge[5] = {6, 4, 8, 2, 6}, kResolve[5] = {8, 4, 16, 8, 2};

static sem_status frame_begin(sem_ctx *ctx, const RenderFrame &F)
{
    // until k_resolve has run, the keys are not all "empty"
    ctx->render_keys_dirty = true;
    // the large-triangle count and the parts' tile counters
    SEM_CU(ctx, cudaMemsetAsync(F.nlarge, 0, sizeof(int32_t) * (1 + RENDER_MAX_PARTS), ctx->stream));
    return SEM_OK;
}

static sem_status frame_end(sem_ctx *ctx, const RenderFrame &F, const float *tris, int w, uint8_t *rgba, float *depth)
{
    if (F.ntri > 0) {
        SEM_TRACED(ctx, "k_raster_large", k_raster_large<<<kLarge[w] * ctx->sm_count, LARGE_THREADS, 0,
                                                           ctx->stream>>>(tris, F.large, F.nlarge, F.P, F.keys));
        SEM_CU(ctx, cudaGetLastError());
    }
    const int64_t rgrid = std::max<int64_t>(1, std::min<int64_t>((F.npx / 4 + 255) / 256,
                                                                 (int64_t)kResolve[w] * ctx->sm_count));
    SEM_TRACED(ctx, "k_resolve", k_resolve<<<(unsigned)rgrid, 256, 0, ctx->stream>>>(
                                     F.colors, F.npx, F.keys, reinterpret_cast<uint32_t *>(rgba), depth));
    SEM_CU(ctx, cudaGetLastError());
    ctx->render_keys_dirty = false;
    return SEM_OK;
}

sem_status render_run(sem_ctx *ctx, const float *tris, int64_t ntri64, const int64_t *seg_ntri, int nseg,
                      const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth,
                      const int64_t *seg_start_dev, unsigned long long seg_mask)
{
    RenderFrame F;
    SEM_TRY(render_setup(ctx, F, ntri64, seg_ntri, nseg, seg_rgb, cam, W, H, seg_start_dev, seg_mask));
    // one frame; the frame leaves the key buffer all "empty" again, so every candidate width of
    // the autotuner draws the same image
    const bool masked = F.P.seg_mask != ~0ull;
    int masked_per_sm = 1;
    if (masked) {
        static KernelSetup ks;
        SEM_TRY(kernel_setup(ctx, ks, k_raster_masked, 256, 0, &masked_per_sm));
    }
    auto frame = [&](int w) -> sem_status {
        SEM_TRY(frame_begin(ctx, F));
        if (F.ntri > 0 && !masked) {
            SEM_TRACED(ctx, "k_raster_small", k_raster_small<<<(F.ntri + 255) / 256, 256, 0, ctx->stream>>>(
                                                  tris, F.ntri, F.P.nseg, F.P, F.keys, F.large, F.nlarge, F.colors));
            SEM_CU(ctx, cudaGetLastError());
        } else if (F.ntri > 0) {
            // a draw mask: only the drawn segments' tiles, from the frame's first tile counter
            const int64_t grid = std::min<int64_t>(((int64_t)F.ntri + 255) / 256 + F.P.nseg,
                                                   (int64_t)masked_per_sm * ctx->sm_count);
            SEM_TRACED(ctx, "k_raster_masked", k_raster_masked<<<(unsigned)grid, 256, 0, ctx->stream>>>(
                                                   tris, F.ntri, F.P, F.keys, F.large, F.nlarge, F.colors,
                                                   F.next_tile));
            SEM_CU(ctx, cudaGetLastError());
        }
        return frame_end(ctx, F, tris, w, rgba, depth);
    };
    static const int kCand[5] = {0, 1, 2, 3, 4};
    return width_tuned(ctx, TUNE_RENDER, W, H, kCand, F.ntri > 0 ? 5 : 1, 0, frame);
}

// ------------------------------------------------------------------------------------------
// A frame drawn in parts (sem_frame_async): begun on the context's stream, its segment ranges
// drawn on whichever stream produced their triangles, ended (large triangles, resolve) on the
// context's stream once every part is ordered before it.  One frame in progress per context.
sem_status render_frame_begin(sem_ctx *ctx, int64_t ntri_max, const int64_t *seg_start_dev, int nseg,
                              const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth)
{
    if (!ctx->frame) ctx->frame = new RenderFrame();
    RenderFrame &F = *ctx->frame;
    std::vector<int64_t> zeros(nseg > 0 ? nseg : 1, 0);
    SEM_TRY(render_setup(ctx, F, ntri_max, zeros.data(), nseg, seg_rgb, cam, W, H, seg_start_dev, ~0ull));
    F.rgba = rgba;
    F.depth = depth;
    return frame_begin(ctx, F);
}

// Segments [seg_lo, seg_hi) of the frame begun last, as its part `part` (each part of a frame
// has its own tile counter), on ctx->stream.
sem_status render_frame_draw(sem_ctx *ctx, const float *tris, int seg_lo, int seg_hi, int part)
{
    if (!ctx->frame) return sem_fail(ctx, SEM_ERR_ARG, "frame draw without a frame begun");
    RenderFrame &F = *ctx->frame;
    if (part < 0 || part >= RENDER_MAX_PARTS) return sem_fail(ctx, SEM_ERR_ARG, "frame part %d", part);
    if (F.ntri <= 0 || seg_lo >= seg_hi) return SEM_OK;
    if (seg_lo == 0) {
        // a part from the buffer's start: one tile per block up to the part's end (blocks past it
        // leave at once), the faster form
        SEM_TRACED(ctx, "k_raster_small", k_raster_small<<<(F.ntri + 255) / 256, 256, 0, ctx->stream>>>(
                                              tris, F.ntri, seg_hi, F.P, F.keys, F.large, F.nlarge, F.colors));
        return sem_cuda(ctx, cudaGetLastError(), "k_raster_small launch");
    }
    static KernelSetup ks;
    int per_sm = 1;
    SEM_TRY(kernel_setup(ctx, ks, k_raster_range, 256, 0, &per_sm));
    const int64_t tiles = ((int64_t)F.ntri + 255) / 256 + 1;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * ctx->sm_count);
    SEM_TRACED(ctx, "k_raster_range", k_raster_range<<<(unsigned)grid, 256, 0, ctx->stream>>>(
                                          tris, F.ntri, seg_lo, seg_hi, F.P, F.keys, F.large, F.nlarge, F.colors,
                                          F.next_tile + part));
    return sem_cuda(ctx, cudaGetLastError(), "k_raster_range launch");
}

// Large triangles and resolve of the frame begun last, on ctx->stream, with the launch widths the
// autotuner chose for this frame size (the defaults when it has not chosen yet).
sem_status render_frame_end(sem_ctx *ctx, const float *tris)
{
    if (!ctx->frame) return sem_fail(ctx, SEM_ERR_ARG, "frame end without a frame begun");
    RenderFrame &F = *ctx->frame;
    int w = 0;
    for (const auto &t : ctx->width_tune)
        if (t.kind == TUNE_RENDER && t.N == F.P.W && t.size == F.P.H) w = t.width;
    return frame_end(ctx, F, tris, w, F.rgba, F.depth);
}

bool render_width_settled(sem_ctx *ctx, int W, int H)
{
    if (!ctx->autotune || ctx->trace_on) return true;
    for (const auto &t : ctx->width_tune)
        if (t.kind == TUNE_RENDER && t.N == W && t.size == H) return true;
    return false;
}

void render_frame_free(sem_ctx *ctx)
{
    delete ctx->frame;
    ctx->frame = nullptr;
}
