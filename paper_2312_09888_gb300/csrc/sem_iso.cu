// sem_iso.cu -- marching-cubes isosurface over the GLL sub-hexes of each element.
//
// Method: Lorensen & Cline 1987, applied to the N^3 sub-hexes of each element's
// (N+1)^3 GLL lattice.  Cell (i,j,k) has corners v = a + 2b + 4c at node (i+a, j+b, k+c);
// case = sum_v [f_v >= iso] 2^v; triangles come from the library's generated case table;
// a cut edge (lo, hi) gets t = (iso - f_lo)/(f_hi - f_lo), p = p_lo + t (p_hi - p_lo).
//
// Three passes over (element, isovalue) units, all isovalues of a field in one read of it:
//   counting     k_iso_count_p (persistent, N <= 9) / k_iso_count_m: one warp per element,
//                node masks by warp ballots, cell classification from node rows, one triangle
//                count per unit (and optionally every cell's case); for Q on N = 7 box meshes
//                the Q kernel itself counts (k_sem_q8<true>, sem_qcrit.cu);
//   scan         k_scan_lookback (sem_scan.cu): exclusive scan of the counts -> each unit's
//                first triangle, and the list of units that hold triangles;
//   emit         k_iso_emit_m: persistent warps take listed units, re-read the element, list its
//                cut cells and write its triangles in (isovalue, element, cell, table) order.
// sem_isosurface_noalloc keeps the one-isovalue kernels k_iso_count / k_iso_emit (one warp per
// element, fixed scratch).  Node positions are lerps of the element box with exact end points,
// so nodes shared by two elements get bit-identical coordinates.
#include <cuda_runtime.h>

#include <algorithm>
#include <string.h>

#include "sem_internal.cuh"

#define MP (SEM_MAX_ORDER + 1)
#define ISO_MAXT 5      // largest triangle count of the generated table (checked on upload)
// elements (warps) per block: 8, fewer for large orders so static shared memory stays < 40 KB
template <int NP>
struct IsoW {
    static constexpr int B = 4 * NP * NP * NP;
    static constexpr int V = (40960 / B) < 1 ? 1 : ((40960 / B) > 8 ? 8 : (40960 / B));
};

__constant__ float c_s[(SEM_MAX_ORDER + 1) * MP];        // (xi+1)/2 per order
__constant__ uint8_t c_ntri[256];
__constant__ int8_t c_edge[256 * ISO_MAXT * 3];
// per (case, triangle): the corner pairs (lo | hi << 3) of its three edges, 6 bits each
__constant__ uint32_t c_tri_corners[256 * ISO_MAXT];

sem_status iso_upload_tables(sem_ctx *ctx, const float *s_all, const int32_t *ntri, const int8_t *edges)
{
    uint8_t n8[256];
    int8_t e8[256 * ISO_MAXT * 3];
    for (int c = 0; c < 256; ++c) {
        if (ntri[c] > ISO_MAXT) return sem_fail(ctx, SEM_ERR_CUDA, "case table has %d triangles", ntri[c]);
        n8[c] = (uint8_t)ntri[c];
        for (int q = 0; q < ISO_MAXT * 3; ++q) e8[c * ISO_MAXT * 3 + q] = edges[c * SEM_MC_MAXT * 3 + q];
    }
    // edge e -> (lower corner, upper corner) in lexicographic edge order
    static const int kLo[12] = {0, 0, 0, 1, 1, 2, 2, 3, 4, 4, 5, 6}, kHi[12] = {1, 2, 4, 3, 5, 3, 6, 7, 5, 6, 7, 7};
    uint32_t tc[256 * ISO_MAXT];
    for (int c = 0; c < 256; ++c)
        for (int t = 0; t < ISO_MAXT; ++t) {
            uint32_t x = 0;
            if (t < ntri[c])
                for (int v = 0; v < 3; ++v) {
                    const int e = e8[(c * ISO_MAXT + t) * 3 + v];
                    if (e < 0 || e > 11) return sem_fail(ctx, SEM_ERR_CUDA, "case table edge %d out of range", e);
                    x |= (uint32_t)(kLo[e] | (kHi[e] << 3)) << (6 * v);
                }
            tc[c * ISO_MAXT + t] = x;
        }
    SEM_CU(ctx, cudaMemcpyToSymbol(c_tri_corners, tc, sizeof tc));
    SEM_CU(ctx, cudaMemcpyToSymbol(c_s, s_all, sizeof(float) * (SEM_MAX_ORDER + 1) * MP));
    SEM_CU(ctx, cudaMemcpyToSymbol(c_ntri, n8, sizeof n8));
    SEM_CU(ctx, cudaMemcpyToSymbol(c_edge, e8, sizeof e8));
    void *nt = nullptr;
    SEM_CU(ctx, cudaGetSymbolAddress(&nt, c_ntri));
    ctx->d_ntri = static_cast<const uint8_t *>(nt);
    return SEM_OK;
}

// edge e -> (lower corner, upper corner), lexicographic numbering
// (0,1)(0,2)(0,4)(1,3)(1,5)(2,3)(2,6)(3,7)(4,5)(4,6)(5,7)(6,7), packed one nibble per edge
__device__ __forceinline__ void edge_ends(int e, int &lo, int &hi)
{
    lo = (int)((0x654432211000ull >> (4 * e)) & 15u);
    hi = (int)((0x776576353421ull >> (4 * e)) & 15u);
}

template <int NP>
__device__ __forceinline__ void load_element(const float *__restrict__ fe, float *__restrict__ sf, int lane, float iso,
                                             bool &any_in, bool &any_out)
{
    constexpr int NP3 = NP * NP * NP;
    bool ai = false, ao = false;
    if constexpr (NP3 % 128 == 0) {
        const float4 *f4 = reinterpret_cast<const float4 *>(fe);
        float4 *s4 = reinterpret_cast<float4 *>(sf);
#pragma unroll
        for (int q = 0; q < NP3 / 128; ++q) {
            float4 v = __ldg(f4 + q * 32 + lane);
            s4[q * 32 + lane] = v;
            ai |= (v.x >= iso) | (v.y >= iso) | (v.z >= iso) | (v.w >= iso);
            ao |= !(v.x >= iso) | !(v.y >= iso) | !(v.z >= iso) | !(v.w >= iso);
        }
    } else {
        for (int idx = lane; idx < NP3; idx += 32) {
            float v = __ldg(fe + idx);
            sf[idx] = v;
            ai |= v >= iso;
            ao |= !(v >= iso);
        }
    }
    any_in = __any_sync(0xffffffffu, ai);
    any_out = __any_sync(0xffffffffu, ao);
}

template <int NP>
__device__ __forceinline__ int cell_case(const float *__restrict__ sf, int c, float iso, int &i, int &j, int &k)
{
    constexpr int N = NP - 1;
    i = c % N;
    j = (c / N) % N;
    k = c / (N * N);
    const int b = (k * NP + j) * NP + i;
    int cs = 0;
    cs |= (sf[b] >= iso) << 0;
    cs |= (sf[b + 1] >= iso) << 1;
    cs |= (sf[b + NP] >= iso) << 2;
    cs |= (sf[b + NP + 1] >= iso) << 3;
    cs |= (sf[b + NP * NP] >= iso) << 4;
    cs |= (sf[b + NP * NP + 1] >= iso) << 5;
    cs |= (sf[b + NP * NP + NP] >= iso) << 6;
    cs |= (sf[b + NP * NP + NP + 1] >= iso) << 7;
    return cs;
}

template <int NP>
__global__ void __launch_bounds__(32 * IsoW<NP>::V) k_iso_count(const float *__restrict__ f, float iso, int64_t E,
                                                             int32_t *__restrict__ elem_cnt, uint8_t *__restrict__ cases)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    __shared__ __align__(16) float s_f[IsoW<NP>::V][NP3];
    __shared__ uint8_t s_nt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * IsoW<NP>::V + w;
    if (e >= E) return;
    float *sf = s_f[w];
    bool any_in, any_out;
    load_element<NP>(f + e * NP3, sf, lane, iso, any_in, any_out);
    if (!(any_in && any_out)) {
        if (lane == 0) elem_cnt[e] = 0;
        if (cases) {
            const uint8_t v = any_in ? 255 : 0;
            for (int c = lane; c < N3; c += 32) cases[e * N3 + c] = v;
        }
        return;
    }
    __syncwarp();
    int cnt = 0;
    for (int c = lane; c < N3; c += 32) {
        int i, j, k;
        const int cs = cell_case<NP>(sf, c, iso, i, j, k);
        cnt += s_nt[cs];
        if (cases) cases[e * N3 + c] = (uint8_t)cs;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if (lane == 0) elem_cnt[e] = cnt;
}

template <int NP>
__global__ void __launch_bounds__(32 * IsoW<NP>::V) k_iso_emit(const float *__restrict__ f, float iso, int64_t E,
                                                            const int64_t *__restrict__ offs,
                                                            const float4 *__restrict__ blo,
                                                            const float4 *__restrict__ bhi, float *__restrict__ tris,
                                                            int32_t *__restrict__ tri_elem, int64_t cap)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    __shared__ __align__(16) float s_f[IsoW<NP>::V][NP3];
    __shared__ uint8_t s_nt[256];
    __shared__ int8_t s_ed[256 * ISO_MAXT * 3];
    __shared__ float s_s[NP];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    for (int t = threadIdx.x; t < 256 * ISO_MAXT * 3; t += blockDim.x) s_ed[t] = c_edge[t];
    if (threadIdx.x < NP) s_s[threadIdx.x] = c_s[(NP - 1) * MP + threadIdx.x];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * IsoW<NP>::V + w;
    if (e >= E) return;
    int64_t base = offs[e];
    if (offs[e + 1] == base) return;
    float *sf = s_f[w];
    bool ai, ao;
    load_element<NP>(f + e * NP3, sf, lane, iso, ai, ao);
    __syncwarp();
    const float4 L = blo[e], H = bhi[e];
    for (int c0 = 0; c0 < N3; c0 += 32) {
        const int c = c0 + lane;
        int cs = 0, nt = 0, i = 0, j = 0, k = 0;
        if (c < N3) {
            cs = cell_case<NP>(sf, c, iso, i, j, k);
            nt = s_nt[cs];
        }
        int incl = nt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int64_t o = base + (incl - nt);
        for (int q = 0; q < nt; ++q, ++o) {
            float p[9];
#pragma unroll
            for (int sv = 0; sv < 3; ++sv) {
                int lo, hi;
                edge_ends(s_ed[(cs * ISO_MAXT + q) * 3 + sv], lo, hi);
                const int ia = i + (lo & 1), ja = j + ((lo >> 1) & 1), ka = k + ((lo >> 2) & 1);
                const int ib = i + (hi & 1), jb = j + ((hi >> 1) & 1), kb = k + ((hi >> 2) & 1);
                const float fa = sf[(ka * NP + ja) * NP + ia], fb = sf[(kb * NP + jb) * NP + ib];
                const float t = (iso - fa) / (fb - fa);
                const float xa = fmaf(s_s[ia], H.x, (1.f - s_s[ia]) * L.x), xb = fmaf(s_s[ib], H.x, (1.f - s_s[ib]) * L.x);
                const float ya = fmaf(s_s[ja], H.y, (1.f - s_s[ja]) * L.y), yb = fmaf(s_s[jb], H.y, (1.f - s_s[jb]) * L.y);
                const float za = fmaf(s_s[ka], H.z, (1.f - s_s[ka]) * L.z), zb = fmaf(s_s[kb], H.z, (1.f - s_s[kb]) * L.z);
                p[sv * 3 + 0] = fmaf(t, xb - xa, xa);
                p[sv * 3 + 1] = fmaf(t, yb - ya, ya);
                p[sv * 3 + 2] = fmaf(t, zb - za, za);
            }
            if (o < cap) {
                float *dst = tris + o * 9;
#pragma unroll
                for (int r = 0; r < 9; ++r) dst[r] = p[r];
                if (tri_elem) tri_elem[o] = (int32_t)e;
            }
        }
        base += total;
    }
}

// ------------------------------------------------------------------------------------------
// Several isovalues at once (sem_isosurface_multi; sem_isosurface is the one-isovalue case).
// The field is read once per pass for all isovalues: each cell's 8 corners are loaded once
// and classified against every isovalue.  Counts are laid out [q][e], so one scan over
// niso*E entries gives every isovalue's triangles a contiguous segment, in isovalue order.
// Emission stages each round's triangles in shared memory and stores them coalesced.

struct IsoSet {
    int niso;
    float iso[SEM_MAX_ISO];
};

// Node masks.  For isovalue q, bit b of word w of the element's mask is [f_n >= iso_q] for node
// n = 32w + b (NaN is never inside).  One warp ballot makes one word, so the masks come out of
// the coalesced load of the element at one vote per 32 nodes and isovalue, and the same votes
// cull the element: it is active for q iff some node is inside and some is not.
template <int NP>
struct MaskGeo {
    static constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N, NRP = N * N;
    static constexpr int NW = (NP3 + 31) / 32;
    static constexpr int MW = NW + 1;  // one zero word of padding for the funnel shift below
};

// Loads element fe (and copies it to sf unless null); writes the masks of all S.niso isovalues
// to m[q * MW + w]; returns the activity bits of the isovalues.
template <int NP>
__device__ __forceinline__ unsigned load_masks(const float *__restrict__ fe, float *__restrict__ sf, const IsoSet &S,
                                               uint32_t *__restrict__ m, int lane)
{
    using G = MaskGeo<NP>;
    // loads in chunks of up to 16 words, all issued before the chunk's votes
    constexpr int CH = G::NW < 16 ? G::NW : 16;
    unsigned any_in = 0, not_all = 0;
    for (int w0 = 0; w0 < G::NW; w0 += CH) {
        float v[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int w = w0 + c, n = w * 32 + lane;
            const bool valid = (G::NW % CH == 0 || w < G::NW) && ((G::NP3 % 32 == 0) || n < G::NP3);
            v[c] = valid ? __ldg(fe + n) : 0.f;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int w = w0 + c, n = w * 32 + lane;
            if (G::NW % CH != 0 && w >= G::NW) break;
            const bool valid = (G::NP3 % 32 == 0) || n < G::NP3;
            if (sf && valid) sf[n] = v[c];
            const uint32_t vmask = (G::NP3 % 32 == 0 || w < G::NW - 1) ? ~0u : ((1u << (G::NP3 % 32)) - 1u);
#pragma unroll
            for (int q = 0; q < SEM_MAX_ISO; ++q) {
                if (q >= S.niso) break;
                const uint32_t b = __ballot_sync(0xffffffffu, valid && v[c] >= S.iso[q]);
                if (lane == 0) m[q * G::MW + w] = b;
                any_in |= (b != 0u ? 1u : 0u) << q;
                not_all |= ((b | ~vmask) != ~0u ? 1u : 0u) << q;
            }
        }
    }
    if (lane < S.niso) m[lane * G::MW + G::NW] = 0u;
    return any_in & not_all;
}

// The NP inside-bits of node row (k, j) (nodes i = 0..N along r).
template <int NP>
__device__ __forceinline__ uint32_t row_bits(const uint32_t *__restrict__ m, int k, int j)
{
    const int o = (k * NP + j) * NP;
    if constexpr (NP == 8) return reinterpret_cast<const uint8_t *>(m)[o >> 3];
    else if constexpr (NP == 16) return reinterpret_cast<const uint16_t *>(m)[o >> 4];
    else return __funnelshift_r(m[o >> 5], m[(o >> 5) + 1], o & 31) & ((1u << NP) - 1u);
}

// Cells (i, j, k), i = 0..N-1, of the row pair (j, k) whose corners are neither all inside nor
// all outside, from the four node rows that bound them.
template <int NP>
__device__ __forceinline__ uint32_t cut_cells(uint32_t r00, uint32_t r01, uint32_t r10, uint32_t r11)
{
    const uint32_t A = r00 & r01 & r10 & r11, O = r00 | r01 | r10 | r11;
    return (O | (O >> 1)) & ~(A & (A >> 1)) & ((1u << (NP - 1)) - 1u);
}

// case of cell i of the row pair: corner v = a + 2b + 4c is bit (i + a) of row (k + c, j + b)
__device__ __forceinline__ int pair_case(uint32_t r00, uint32_t r01, uint32_t r10, uint32_t r11, int i)
{
    return (int)(((r00 >> i) & 3u) | (((r01 >> i) & 3u) << 2) | (((r10 >> i) & 3u) << 4) | (((r11 >> i) & 3u) << 6));
}

#define COUNT_WARPS 8

// The element's values for the register-held masks below: lane l holds nodes 32 w + l.
template <int NP>
__device__ __forceinline__ void load_vals(const float *__restrict__ fe, float (&v)[MaskGeo<NP>::NW], int lane)
{
    using G = MaskGeo<NP>;
#pragma unroll
    for (int w = 0; w < G::NW; ++w) {
        const int n = w * 32 + lane;
        v[w] = ((G::NP3 % 32 == 0) || n < G::NP3) ? __ldg(fe + n) : 0.f;
    }
}

// The masks of all isovalues of an element from its register-held values: lane w keeps mask
// word w of each isovalue and stores it; the activity bits come from warp AND/OR reductions
// of the words.  For orders with at most 32 mask words (N <= 9).
template <int NP>
__device__ __forceinline__ unsigned masks_from_vals(const float (&v)[MaskGeo<NP>::NW], const IsoSet &S,
                                                    uint32_t *__restrict__ m, int lane)
{
    using G = MaskGeo<NP>;
    static_assert(G::NW <= 32, "one mask word per lane");
    // lanes >= NW hold the neutral words of the reductions (AND: all ones, OR: zero)
    const uint32_t vmask = lane >= G::NW ? 0u
                           : (G::NP3 % 32 == 0 || lane < G::NW - 1) ? ~0u
                                                                     : ((1u << (G::NP3 % 32)) - 1u);
    unsigned active = 0;
#pragma unroll
    for (int q = 0; q < SEM_MAX_ISO; ++q) {
        if (q >= S.niso) break;
        uint32_t mine = 0;
#pragma unroll
        for (int w = 0; w < G::NW; ++w) {
            const int n = w * 32 + lane;
            const bool valid = (G::NP3 % 32 == 0) || n < G::NP3;
            const uint32_t b = __ballot_sync(0xffffffffu, valid && v[w] >= S.iso[q]);
            if (lane == w) mine = b;
        }
        if (lane < G::NW) m[q * G::MW + lane] = mine;
        if (lane == G::NW) m[q * G::MW + lane] = 0u;  // padding word
        const uint32_t any_in = __reduce_or_sync(0xffffffffu, mine & vmask);
        const uint32_t all_in = __reduce_and_sync(0xffffffffu, mine | ~vmask);
        if (any_in != 0u && all_in != ~0u) active |= 1u << q;
    }
    return active;
}

template <int NP>
__device__ __forceinline__ unsigned load_masks_reg(const float *__restrict__ fe, const IsoSet &S,
                                                   uint32_t *__restrict__ m, int lane)
{
    float v[MaskGeo<NP>::NW];
    load_vals<NP>(fe, v, lane);
    return masks_from_vals<NP>(v, S, m, lane);
}

// Triangle counts of element e for every isovalue from its masks (and every cell's case when
// `cases` is not null).
template <int NP>
__device__ __forceinline__ void count_element(const uint32_t *__restrict__ m, unsigned active, const IsoSet &S,
                                              int64_t e, int64_t E, const uint8_t *__restrict__ s_nt,
                                              int32_t *__restrict__ cnt, uint8_t *__restrict__ cases, int lane)
{
    using G = MaskGeo<NP>;
    constexpr int N = G::N, N3 = G::N3, MW = G::MW;
    for (int q = 0; q < S.niso; ++q) {
        const uint32_t *mq = m + q * MW;
        if (!((active >> q) & 1u)) {
            if (lane == 0) cnt[q * E + e] = 0;
            if (cases) {
                const uint8_t v = (mq[0] & 1u) ? 255 : 0;  // every node on the same side as node 0
                for (int c = lane; c < N3; c += 32) cases[(q * E + e) * N3 + c] = v;
            }
            continue;
        }
        int acc = 0;
        for (int rp = lane; rp < G::NRP; rp += 32) {
            const int j = rp % N, k = rp / N;
            const uint32_t r00 = row_bits<NP>(mq, k, j), r01 = row_bits<NP>(mq, k, j + 1);
            const uint32_t r10 = row_bits<NP>(mq, k + 1, j), r11 = row_bits<NP>(mq, k + 1, j + 1);
            if (cases)
                for (int i = 0; i < N; ++i) cases[(q * E + e) * N3 + i + N * rp] = (uint8_t)pair_case(r00, r01, r10, r11, i);
            for (uint32_t act = cut_cells<NP>(r00, r01, r10, r11); act; act &= act - 1u)
                acc += s_nt[pair_case(r00, r01, r10, r11, __ffs(act) - 1)];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == 0) cnt[q * E + e] = acc;
    }
}

// One warp per element.
template <int NP>
__global__ void __launch_bounds__(32 * COUNT_WARPS) k_iso_count_m(const float *__restrict__ f,
                                                                 const __grid_constant__ IsoSet S, int64_t E,
                                                                 int32_t *__restrict__ cnt, uint8_t *__restrict__ cases)
{
    using G = MaskGeo<NP>;
    __shared__ uint32_t s_m[COUNT_WARPS][SEM_MAX_ISO * G::MW];
    __shared__ uint8_t s_nt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * COUNT_WARPS + w;
    if (e >= E) return;
    uint32_t *m = s_m[w];
    unsigned active;
    if constexpr (G::NW <= 32) active = load_masks_reg<NP>(f + e * G::NP3, S, m, lane);
    else active = load_masks<NP>(f + e * G::NP3, nullptr, S, m, lane);
    __syncwarp();
    count_element<NP>(m, active, S, e, E, s_nt, cnt, cases, lane);
}

// Persistent form for orders with at most 32 mask words (N <= 9): warps stride over the
// elements, and each issues the loads of its next element before it classifies the current
// one, so two elements per warp are in flight and no block is launched per 8 elements.  The
// grid is one resident wave (SMs x blocks per SM).
template <int NP>
__global__ void __launch_bounds__(32 * COUNT_WARPS) k_iso_count_p(const float *__restrict__ f,
                                                                 const __grid_constant__ IsoSet S, int64_t E,
                                                                 int32_t *__restrict__ cnt, uint8_t *__restrict__ cases)
{
    using G = MaskGeo<NP>;
    __shared__ uint32_t s_m[COUNT_WARPS][SEM_MAX_ISO * G::MW];
    __shared__ uint8_t s_nt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * COUNT_WARPS;
    int64_t e = (int64_t)blockIdx.x * COUNT_WARPS + w;
    if (e >= E) return;
    uint32_t *m = s_m[w];
    float v[G::NW];
    load_vals<NP>(f + e * G::NP3, v, lane);
    for (; e < E; e += stride) {
        float nv[G::NW];
        const int64_t en = e + stride;
        if (en < E) load_vals<NP>(f + en * G::NP3, nv, lane);
        __syncwarp();  // the previous element's readers of m are done
        const unsigned active = masks_from_vals<NP>(v, S, m, lane);
        __syncwarp();
        count_element<NP>(m, active, S, e, E, s_nt, cnt, cases, lane);
        if (en < E) {
#pragma unroll
            for (int q = 0; q < G::NW; ++q) v[q] = nv[q];
        }
    }
}

// Launch of the counting pass: the persistent kernel for N <= 9, else one warp per element.
template <int NP>
static sem_status launch_count(sem_ctx *ctx, const float *f, const IsoSet &S, int64_t E, int32_t *cnt,
                               uint8_t *cases)
{
    if constexpr (MaskGeo<NP>::NW <= 32) {
        static KernelSetup ks;  // per instantiation and device
        int per_sm = 1;
        SEM_TRY(kernel_setup(ctx, ks, k_iso_count_p<NP>, 32 * COUNT_WARPS, 0, &per_sm));
        int64_t grid = (int64_t)ctx->sm_count * per_sm;
        const int64_t need = (E + COUNT_WARPS - 1) / COUNT_WARPS;
        if (grid > need) grid = need;
        SEM_TRACED(ctx, "k_iso_count_p", k_iso_count_p<NP><<<(unsigned)grid, 32 * COUNT_WARPS, 0, ctx->stream>>>(
            f, S, E, cnt, cases));
    } else {
        SEM_TRACED(ctx, "k_iso_count_m", k_iso_count_m<NP><<<(unsigned)((E + COUNT_WARPS - 1) / COUNT_WARPS),
                                                            32 * COUNT_WARPS, 0, ctx->stream>>>(f, S, E, cnt, cases));
    }
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_count launch");
}

// per-warp dynamic shared memory of the emit kernel: the element's field, a window of the
// triangle map, the mask of one isovalue, the element's node coordinates, a store staging area
// and the list of cut cells; warps per block: up to 8 within ~96 KB
#define EMIT_MAPCAP 256  // map window: triangles of one (element, isovalue) handled per pass
#define EMIT_UNITS_DEFAULT 1  // units with triangles a warp takes per atomic, untuned
#define EMIT_MINB 4  // resident blocks per SM the register allocation is sized for (64 registers a thread)
template <int NP>
struct EmitW {
    using G = MaskGeo<NP>;
    static constexpr int r16(int b) { return ((b + 15) / 16) * 16; }
    static constexpr int F_BYTES = r16(4 * G::NP3);
    static constexpr int MAP_BYTES = 4 * EMIT_MAPCAP;
    static constexpr int M_BYTES = r16(4 * G::MW);
    static constexpr int X_BYTES = r16(4 * 3 * NP);
    static constexpr int STG_BYTES = 32 * 9 * 4;
    static constexpr int LIST_BYTES = r16(4 * G::N3);  // the element's cut cells: cell | case << 16
    static constexpr int B = F_BYTES + MAP_BYTES + M_BYTES + X_BYTES + STG_BYTES + LIST_BYTES;
    static constexpr int R = 98304 / B;
    static constexpr int V = R < 1 ? 1 : (R > 8 ? 8 : R);
};

// node offset of corner v = a + 2b + 4c from the cell's corner 0
template <int NP>
__device__ __forceinline__ int corner_off(int v)
{
    return (v & 1) + ((v >> 1) & 1) * NP + (v >> 2) * NP * NP;
}

// Per-warp shared memory of the emit kernel (see EmitW).
struct EmitSmem {
    float *sf;      // the element's field
    uint32_t *map;  // cs << 16 | k << 12 | j << 8 | i << 4 | t
    uint32_t *m;    // the unit's node mask
    float *X, *Y, *Z;
    float *stg;
    uint32_t *list;  // cut cells: cell | case << 16
};

// One (element, isovalue) unit u = q E + e with n > 0 triangles from tris[o]: load the element
// and its mask for the unit's isovalue, then (1a) lane per row pair, list the cut cells with their cases in cell order (a warp scan of the per-lane
// counts places each lane's run; N uniform passes over the cells of a row, each cut cell stored
// at its rank, so no lane walks its cells alone); then per window of EMIT_MAPCAP triangles (1b)
// lane per listed cell, warp-scan the triangle counts and write each triangle's packed (case,
// cell, index in cell) into the map, in cell order; (2) lane per output triangle: interpolate
// its three vertices and stage them, then store each round of 32 triangles (1152 contiguous
// bytes) with coalesced 4-byte stores.  On a box mesh the lerp between the edge's two node
// positions is taken per axis from the cell's corner coordinates: x_lo + t (x_hi - x_lo) along
// the edge's axis, x + t 0 along the other two (the same FP32 operations as the lerp of the two
// nodes, whose other coordinates agree); on a general mesh it is the lerp between the two
// nodes' own coordinates.
template <int NP, bool GENERAL>
__device__ __forceinline__ void emit_unit(const float *__restrict__ f, const IsoSet &S, int64_t E, int64_t u, int64_t o, int64_t n,
                                          const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                                          float *__restrict__ tris, int32_t *__restrict__ tri_elem,
                                          const float *__restrict__ xyzn, const EmitSmem &sm,
                                          const uint8_t *__restrict__ s_nt, const uint32_t *__restrict__ s_tc,
                                          const float *__restrict__ s_s, int lane)
{
    using G = MaskGeo<NP>;
    constexpr int N = G::N;
    const int q = (int)(u / E);
    const int64_t e = u - (int64_t)q * E;
    const float iso = S.iso[q];
    float *sf = sm.sf, *X = sm.X, *Y = sm.Y, *Z = sm.Z, *stg = sm.stg;
    uint32_t *map = sm.map, *m = sm.m, *list = sm.list;
    __syncwarp();  // the previous unit's readers of sf, m and X are done
    {
        IsoSet S1;  // the unit's isovalue alone
        S1.niso = 1;
        S1.iso[0] = iso;
        load_masks<NP>(f + e * G::NP3, sf, S1, m, lane);
    }
    if (lane < NP) {
        // node coordinates: lerps of the element box with exact end points
        const float4 L = blo[e], H = bhi[e];
        const float s = s_s[lane];
        X[lane] = fmaf(s, H.x, (1.f - s) * L.x);
        Y[lane] = fmaf(s, H.y, (1.f - s) * L.y);
        Z[lane] = fmaf(s, H.z, (1.f - s) * L.z);
    }
    __syncwarp();
    // (1a) the cut cells of the element, in cell order, with their cases
    int ncells = 0;
    for (int rp0 = 0; rp0 < G::NRP; rp0 += 32) {
        const int rp = rp0 + lane;
        uint32_t act = 0, r00 = 0, r01 = 0, r10 = 0, r11 = 0;
        if (rp < G::NRP) {
            const int j = rp % N, k = rp / N;
            r00 = row_bits<NP>(m, k, j);
            r01 = row_bits<NP>(m, k, j + 1);
            r10 = row_bits<NP>(m, k + 1, j);
            r11 = row_bits<NP>(m, k + 1, j + 1);
            act = cut_cells<NP>(r00, r01, r10, r11);
        }
        const int na = __popc(act);
        int incl = na;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const int at = ncells + incl - na;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((act >> i) & 1u)
                list[at + __popc(act & ((1u << i) - 1u))] =
                    (uint32_t)(rp * N + i) | ((uint32_t)pair_case(r00, r01, r10, r11, i) << 16);
        ncells += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    for (int64_t win = 0; win < n; win += EMIT_MAPCAP) {
        // (1b) the map entries of triangles win .. win + EMIT_MAPCAP - 1, in cell order
        int running = 0;
        for (int c0 = 0; c0 < ncells && running < win + EMIT_MAPCAP; c0 += 32) {
            const int c = c0 + lane;
            const uint32_t ent = c < ncells ? list[c] : 0u;
            const int cs = (int)(ent >> 16);
            const int nt = c < ncells ? s_nt[cs] : 0;
            int incl = nt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            int slot = running + incl - nt - (int)win;
            if (nt > 0) {
                const int cell = (int)(ent & 0xFFFFu), i = cell % N, rp = cell / N;
                const uint32_t key = ((uint32_t)cs << 16) | ((uint32_t)(rp / N) << 12) | ((uint32_t)(rp % N) << 8) |
                                     ((uint32_t)i << 4);
                for (int t = 0; t < nt; ++t, ++slot)
                    if (slot >= 0 && slot < EMIT_MAPCAP) map[slot] = key | (uint32_t)t;
            }
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        // (2) one output triangle per lane, stored through the staging area
        const int cnt = (int)min((int64_t)EMIT_MAPCAP, n - win);
        for (int base = 0; base < cnt; base += 32) {
            const int idx = base + lane;
            if (idx < cnt) {
                const uint32_t key = map[idx];
                const int t = key & 15, i = (key >> 4) & 15, j = (key >> 8) & 15, k = (key >> 12) & 15;
                const int cs = key >> 16;
                const int c0 = (k * NP + j) * NP + i;
                const uint32_t pairs = s_tc[cs * ISO_MAXT + t];
                float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f, z0 = 0.f, z1 = 0.f;
                if constexpr (!GENERAL) {
                    x0 = X[i];
                    x1 = X[i + 1];
                    y0 = Y[j];
                    y1 = Y[j + 1];
                    z0 = Z[k];
                    z1 = Z[k + 1];
                }
                const float dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
#pragma unroll
                for (int sv = 0; sv < 3; ++sv) {
                    const int la = (pairs >> (6 * sv)) & 7, lb = (pairs >> (6 * sv + 3)) & 7;
                    const int na = c0 + corner_off<NP>(la), nb = c0 + corner_off<NP>(lb);
                    const float fa = sf[na], fb = sf[nb];
                    const float tt = __fdividef(iso - fa, fb - fa);
                    if constexpr (GENERAL) {
                        // general mesh: between the two nodes' own coordinates
                        const int64_t tot = E * G::NP3, ga = e * G::NP3 + na, gb = e * G::NP3 + nb;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float pa = __ldg(xyzn + c * tot + ga), pb = __ldg(xyzn + c * tot + gb);
                            stg[lane * 9 + sv * 3 + c] = fmaf(tt, pb - pa, pa);
                        }
                    } else {
                        // the edge runs along the one axis where its corners differ (lo has 0
                        // there); the other axes take a zero step, so a NaN t still makes every
                        // coordinate NaN, as the lerp does
                        const int ax = la ^ lb;
                        stg[lane * 9 + sv * 3 + 0] = fmaf(tt, ax == 1 ? dx : 0.f, (la & 1) ? x1 : x0);
                        stg[lane * 9 + sv * 3 + 1] = fmaf(tt, ax == 2 ? dy : 0.f, (la & 2) ? y1 : y0);
                        stg[lane * 9 + sv * 3 + 2] = fmaf(tt, ax == 4 ? dz : 0.f, (la & 4) ? z1 : z0);
                    }
                }
                if (tri_elem) tri_elem[o + win + idx] = (int32_t)e;
            }
            __syncwarp();
            const int nflt = 9 * min(32, cnt - base);
            float *dst = tris + (o + win + base) * 9;
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const int g = r * 32 + lane;
                if (g < nflt) __stcs(dst + g, stg[g]);  // streamed: read once, by the raster
            }
            __syncwarp();
        }
    }
}

// The units with triangles, live[0 .. nlive) (nlive = next[1], both written by the scan), are
// dealt to persistent warps `units` at a time from the work counter next[0], which the host
// zeroes before the launch; warps therefore hold units with triangles only and finish within
// one unit of each other.  The next counter value is fetched one chunk ahead, and the next
// unit's index and offsets are loaded while the current unit is processed.
template <int NP, bool GENERAL>
__global__ void __launch_bounds__(32 * EmitW<NP>::V, EMIT_MINB) k_iso_emit_m(const float *__restrict__ f,
                                                                 const __grid_constant__ IsoSet S, int64_t E,
                                                                 const int64_t *__restrict__ offs,
                                                                 const int64_t *__restrict__ live,
                                                                 const float4 *__restrict__ blo,
                                                                 const float4 *__restrict__ bhi,
                                                                 float *__restrict__ tris,
                                                                 int32_t *__restrict__ tri_elem, int64_t cap,
                                                                 int *flag, unsigned long long *__restrict__ next,
                                                                 int units, const float *__restrict__ xyzn,
                                                                 const int64_t *__restrict__ base)
{
    using EW = EmitW<NP>;
    const int64_t U = (int64_t)S.niso * E;
    // index of the first triangle in `tris`: 0, or (appending behind an earlier call's
    // segments) a value another kernel wrote on the device
    const int64_t b0 = base ? *base : 0;
    // all-or-nothing capacity check (the host-synchronised path has checked already)
    if (b0 + offs[U] > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && flag) atomicOr(flag, 1 << SEM_ERR_CAPACITY);
        return;
    }
    const int64_t nlive = (int64_t)next[1];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ uint8_t s_nt[256];
    __shared__ uint32_t s_tc[256 * ISO_MAXT];
    __shared__ float s_s[NP];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    for (int t = threadIdx.x; t < 256 * ISO_MAXT; t += blockDim.x) s_tc[t] = c_tri_corners[t];
    if (threadIdx.x < NP) s_s[threadIdx.x] = c_s[(NP - 1) * MP + threadIdx.x];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *mine = s_dyn + (size_t)w * EW::B;
    EmitSmem sm;
    sm.sf = reinterpret_cast<float *>(mine);
    sm.map = reinterpret_cast<uint32_t *>(mine + EW::F_BYTES);
    sm.m = reinterpret_cast<uint32_t *>(mine + EW::F_BYTES + EW::MAP_BYTES);
    sm.X = reinterpret_cast<float *>(mine + EW::F_BYTES + EW::MAP_BYTES + EW::M_BYTES);
    sm.Y = sm.X + NP;
    sm.Z = sm.X + 2 * NP;
    sm.stg = reinterpret_cast<float *>(mine + EW::F_BYTES + EW::MAP_BYTES + EW::M_BYTES + EW::X_BYTES);
    sm.list = reinterpret_cast<uint32_t *>(mine + EW::B - EW::LIST_BYTES);

    // positions in the live list: the chunk [cur, end) in use and, on lane 0, the counter value
    // of the chunk after it (fetched when this one was taken)
    int64_t cur = 0, end = 0;
    unsigned long long ahead = 0;
    bool done = false;
    if (lane == 0) ahead = atomicAdd(next, (unsigned long long)units);
    auto next_pos = [&]() -> int64_t {
        if (cur == end && !done) {
            const int64_t c0 = (int64_t)__shfl_sync(0xffffffffu, ahead, 0);
            if (c0 >= nlive) {
                done = true;
            } else {
                cur = c0;
                end = min(c0 + (int64_t)units, nlive);
                if (lane == 0) ahead = atomicAdd(next, (unsigned long long)units);
            }
        }
        return done ? -1 : cur++;
    };
    const int64_t p0 = next_pos();
    if (p0 < 0) return;
    int64_t u0 = live[p0];
    int64_t o0 = offs[u0], n0 = offs[u0 + 1] - o0;
    const int64_t p1 = next_pos();
    int64_t u1 = p1 >= 0 ? live[p1] : -1;
    for (;;) {
        // ahead of the current unit u0: u1's offsets, u2's index
        int64_t o1 = 0, n1 = 0, u2 = -1;
        if (u1 >= 0) {
            const int64_t p2 = next_pos();
            if (p2 >= 0) u2 = live[p2];
            o1 = offs[u1];
            n1 = offs[u1 + 1] - o1;
        }
        if (b0 + o0 + n0 <= cap)  // holds for every unit after the check above
            emit_unit<NP, GENERAL>(f, S, E, u0, b0 + o0, n0, blo, bhi, tris, tri_elem, xyzn, sm, s_nt, s_tc, s_s, lane);
        if (u1 < 0) break;
        u0 = u1;
        o0 = o1;
        n0 = n1;
        u1 = u2;
    }
}

template <int NP, bool GENERAL>
static sem_status launch_emit_k(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, const int64_t *offs,
                                const int64_t *live, float *tris, int32_t *tri_elem, int64_t cap,
                                unsigned long long *next, int units, const int64_t *base)
{
    constexpr int EV = EmitW<NP>::V;
    constexpr size_t dyn = (size_t)EV * EmitW<NP>::B;
    auto kern = k_iso_emit_m<NP, GENERAL>;
    static KernelSetup ks;  // per instantiation and device
    int blocks_per_sm = 1;
    SEM_TRY(kernel_setup(ctx, ks, kern, 32 * EV, dyn, &blocks_per_sm));
    SEM_CU(ctx, cudaMemsetAsync(next, 0, sizeof(unsigned long long), ctx->stream));
    const unsigned grid = (unsigned)(ctx->sm_count * blocks_per_sm);
    SEM_TRACED(ctx, "k_iso_emit_m", kern<<<grid, 32 * EV, dyn, ctx->stream>>>(f, S, m->E, offs, live, m->lo, m->hi, tris,
                                                                             tri_elem, cap, ctx->d_flag, next, units,
                                                                             m->xyzn, base));
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_emit_m launch");
}

// Launch the persistent emit kernel: one resident wave (SMs x blocks per SM), work counter
// `next` zeroed first; box meshes and general meshes have their own instantiation.
template <int NP>
static sem_status launch_emit(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, const int64_t *offs,
                              const int64_t *live, float *tris, int32_t *tri_elem, int64_t cap,
                              unsigned long long *next, int units, const int64_t *base)
{
    if (m->curved) return launch_emit_k<NP, true>(ctx, m, f, S, offs, live, tris, tri_elem, cap, next, units, base);
    return launch_emit_k<NP, false>(ctx, m, f, S, offs, live, tris, tri_elem, cap, next, units, base);
}

// The emit launch with the context's autotuner: the first emitting call of a given (order,
// elements, isovalues) runs 1, 2, 4 and 8 units per work-counter atomic, each once untimed and
// three times timed with CUDA events (a candidate's time is its fastest run), and keeps the
// fastest; later calls reuse it.  Every candidate writes
// the same triangles to the same places, so the output does not depend on the choice.  Under
// stream capture, or with tuning off, EMIT_UNITS_DEFAULT.
template <int NP>
static sem_status emit(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, const int64_t *offs,
                       const int64_t *live, float *tris, int32_t *tri_elem, int64_t cap, unsigned long long *next,
                       const int64_t *base = nullptr)
{
    for (const auto &t : ctx->emit_tune)
        if (t.N == m->N && t.E == m->E && t.niso == S.niso)
            return launch_emit<NP>(ctx, m, f, S, offs, live, tris, tri_elem, cap, next, t.units, base);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (!ctx->autotune || cs != cudaStreamCaptureStatusNone)
        return launch_emit<NP>(ctx, m, f, S, offs, live, tris, tri_elem, cap, next, EMIT_UNITS_DEFAULT, base);
    cudaEvent_t e0, e1;
    SEM_CU(ctx, cudaEventCreate(&e0));
    SEM_CU(ctx, cudaEventCreate(&e1));
    int best = EMIT_UNITS_DEFAULT;
    float best_ms = 1e30f;
    sem_status st = SEM_OK;
    for (int units : {1, 2, 4, 8}) {
        // once untimed, then three timed runs; the candidate's time is its fastest
        float cand_ms = 1e30f;
        for (int rep = 0; rep < 4 && st == SEM_OK; ++rep) {
            if (rep > 0) st = sem_cuda(ctx, cudaEventRecord(e0, ctx->stream), "event");
            if (st == SEM_OK) st = launch_emit<NP>(ctx, m, f, S, offs, live, tris, tri_elem, cap, next, units, base);
            if (rep > 0 && st == SEM_OK) st = sem_cuda(ctx, cudaEventRecord(e1, ctx->stream), "event");
            if (rep > 0 && st == SEM_OK) st = sem_cuda(ctx, cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            if (rep > 0 && st == SEM_OK) st = sem_cuda(ctx, cudaEventElapsedTime(&ms, e0, e1), "event");
            if (rep > 0 && st == SEM_OK && ms < cand_ms) cand_ms = ms;
        }
        if (st != SEM_OK) break;
        if (cand_ms < best_ms) {
            best_ms = cand_ms;
            best = units;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SEM_TRY(st);
    ctx->emit_tune.push_back({m->N, S.niso, m->E, best, best_ms});
    return SEM_OK;  // the triangles of the last candidate, the same as every other's
}

// Segment ends of an appending call: counts_dev[0] (written earlier on the device) is the first
// triangle's index, counts_dev[q] = counts_dev[0] + offs[q E] for q = 1..niso.
__global__ void k_seg_ends(const int64_t *__restrict__ offs, int64_t E, int niso, int64_t *__restrict__ counts_dev)
{
    const int q = threadIdx.x + 1;
    if (q <= niso) counts_dev[q] = counts_dev[0] + offs[(int64_t)q * E];
}

// The library scratch of one isosurface pass: counts [q][e], offsets, the emit work counter
// (next[0]) and the number of units with triangles (next[1]), the list of those units and the
// scan state.
struct IsoScratch {
    int32_t *cnt;
    int64_t *offs;
    unsigned long long *next;
    int64_t *live;
    void *tmp;
};

static size_t iso_scratch_bytes(int64_t n, size_t &cnt_bytes, size_t &off_bytes, size_t &live_bytes)
{
    cnt_bytes = ((sizeof(int32_t) * n + 255) / 256) * 256;
    off_bytes = ((sizeof(int64_t) * (n + 1) + 255) / 256) * 256;
    live_bytes = ((sizeof(int64_t) * n + 255) / 256) * 256;
    return cnt_bytes + off_bytes + 256 + live_bytes + scan_live_tmp_bytes(n);
}

static void iso_scratch_carve(void *scr, int64_t n, IsoScratch &X)
{
    size_t cb, ob, lb;
    iso_scratch_bytes(n, cb, ob, lb);
    char *p = reinterpret_cast<char *>(scr);
    X.cnt = reinterpret_cast<int32_t *>(p);
    X.offs = reinterpret_cast<int64_t *>(p + cb);
    X.next = reinterpret_cast<unsigned long long *>(p + cb + ob);
    X.live = reinterpret_cast<int64_t *>(p + cb + ob + 256);
    X.tmp = p + cb + ob + 256 + lb;
}

static sem_status iso_scratch_async(sem_ctx *ctx, int64_t n, IsoScratch &X, int arena = SCR_ISO)
{
    size_t cb, ob, lb;
    void *scr;
    SEM_TRY(sem_scratch_nogrow_in_capture(ctx, arena, iso_scratch_bytes(n, cb, ob, lb), &scr));
    iso_scratch_carve(scr, n, X);
    return SEM_OK;
}

template <int NP>
static sem_status iso_multi_np(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, float *tris,
                               int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    const int64_t E = m->E, n = E * S.niso;
    size_t cb, ob, lb;
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_ISO, iso_scratch_bytes(n, cb, ob, lb), &scr));
    IsoScratch X;
    iso_scratch_carve(scr, n, X);
    SEM_TRY(launch_count<NP>(ctx, f, S, E, X.cnt, cases));
    SEM_TRY(scan_i32_i64_live(ctx, X.cnt, X.offs, n, X.tmp, X.live, X.next + 1));
    // segment starts offs[q*E], q = 0..niso (the last one is the grand total)
    SEM_CU(ctx, cudaMemcpy2DAsync(ctx->h_pinned, sizeof(int64_t), X.offs, sizeof(int64_t) * E, sizeof(int64_t),
                                  S.niso + 1, cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < S.niso; ++q) ntri_out[q] = ctx->h_pinned[q + 1] - ctx->h_pinned[q];
    const int64_t total = ctx->h_pinned[S.niso];
    if (!tris) return SEM_OK;  // count-only query
    if (total > cap)
        return sem_fail(ctx, SEM_ERR_CAPACITY, "sem_isosurface: %lld triangles exceed capacity %lld", (long long)total,
                        (long long)cap);
    if (total == 0) return SEM_OK;
    return emit<NP>(ctx, m, f, S, X.offs, X.live, tris, tri_elem, cap, X.next);
}

// Segment starts of a pass whose offsets are in offs: counts_dev[q] = offs[q E] for q = 0..niso,
// or, appending, counts_dev[q] = counts_dev[0] + offs[q E] for q = 1..niso (counts_dev[0], the
// index in tris of the pass's first triangle, an input written earlier on the device).
static sem_status iso_segments_async(sem_ctx *ctx, int64_t E, int niso, const int64_t *offs, int64_t *counts_dev,
                                     bool append)
{
    if (append) {
        SEM_TRACED(ctx, "k_seg_ends", k_seg_ends<<<1, 32, 0, ctx->stream>>>(offs, E, niso, counts_dev));
        return sem_cuda(ctx, cudaGetLastError(), "k_seg_ends launch");
    }
    SEM_CU(ctx, cudaMemcpy2DAsync(counts_dev, sizeof(int64_t), offs, sizeof(int64_t) * E, sizeof(int64_t), niso + 1,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    return SEM_OK;
}

static sem_status iso_scan_async(sem_ctx *ctx, int64_t n, const IsoScratch &X)
{
    return scan_i32_i64_live(ctx, X.cnt, X.offs, n, X.tmp, X.live, X.next + 1);
}

// From the counts on: scan, segment starts to counts_dev, emit.  With `append`, counts_dev[0] is
// an input (the first triangle's index in tris) and only counts_dev[1..niso] are written.
template <int NP>
static sem_status iso_tail_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S,
                                 const IsoScratch &X, float *tris, int32_t *tri_elem, int64_t cap,
                                 int64_t *counts_dev, bool append)
{
    SEM_TRY(iso_scan_async(ctx, m->E * S.niso, X));
    SEM_TRY(iso_segments_async(ctx, m->E, S.niso, X.offs, counts_dev, append));
    if (!tris) return SEM_OK;
    return emit<NP>(ctx, m, f, S, X.offs, X.live, tris, tri_elem, cap, X.next, append ? counts_dev : nullptr);
}

// No host synchronisation: segment starts go to counts_dev (device), a capacity overflow
// raises the context's device flag and writes no triangle.
template <int NP>
static sem_status iso_multi_async_np(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, float *tris,
                                     int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases, bool append)
{
    IsoScratch X;
    SEM_TRY(iso_scratch_async(ctx, m->E * S.niso, X));
    SEM_TRY(launch_count<NP>(ctx, f, S, m->E, X.cnt, cases));
    return iso_tail_async<NP>(ctx, m, f, S, X, tris, tri_elem, cap, counts_dev, append);
}

// Q and its isosurfaces with the counting pass fused into the Q kernel (N = 7 box meshes): the
// Q kernel writes Q and every element's triangle counts, then scan and emit as above.  Other
// meshes run the Q kernel and the isosurface passes one after the other (same results).
sem_status iso_run_q_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                                 float *Q, const float *isos, int niso, float *tris, int32_t *tri_elem, int64_t cap,
                                 int64_t *counts_dev)
{
    if (m->N != 7 || m->curved) {
        SEM_TRY(qcrit_launch(ctx, m, u, v, w, Q));
        return iso_run_multi_async(ctx, m, Q, isos, niso, tris, tri_elem, cap, counts_dev, nullptr, false);
    }
    IsoSet S;
    memset(&S, 0, sizeof S);
    S.niso = niso;
    for (int q = 0; q < niso; ++q) S.iso[q] = isos[q];
    IsoScratch X;
    SEM_TRY(iso_scratch_async(ctx, m->E * S.niso, X));
    SEM_TRY(qcrit_count_launch(ctx, m, u, v, w, Q, niso, isos, X.cnt));
    return iso_tail_async<8>(ctx, m, Q, S, X, tris, tri_elem, cap, counts_dev, false);
}

// ------------------------------------------------------------------------------------------
// Q, its isosurfaces and the isosurfaces of further fields in one call, the further fields'
// passes on the context's auxiliary stream (sem_qcriterion_isosurface_fields_async).
//
//   stream:  Q kernel (+ Q's counts) -> fork -> Q scan, Q segments -> ev_qseg -> Q emit -> join
//   aux:                                fork -> per field k: count, scan, [wait ev_qseg],
//                                               segments (appending), emit -> ev_join
//
// Field k's segments start where field k-1's (or Q's) end, a value written on the device, so
// only the first field's append waits for Q; its counting and scan start with Q's scan.  The
// results are those of the same passes run one after the other.  (A fork before the Q kernel,
// with the first field counted by a slim kernel in the registers and shared memory the Q kernel
// leaves on each SM, was slower: four warps per SM count too slowly, and they slow the Q kernel.)

// true when the emit autotuner has a choice for (order, elements, isovalues), or will not time one
static bool emit_settled(sem_ctx *ctx, const sem_mesh *m, int niso)
{
    if (!ctx->autotune) return true;
    for (const auto &t : ctx->emit_tune)
        if (t.N == m->N && t.E == m->E && t.niso == niso) return true;
    return false;
}

static sem_status aux_ready(sem_ctx *ctx)
{
    if (ctx->aux) return SEM_OK;
    int prio = 0;  // the context stream's priority (the legacy default stream's: 0)
    if (ctx->stream && cudaStreamGetPriority(ctx->stream, &prio) != cudaSuccess) {
        cudaGetLastError();  // not an error of the call: clear it so later launch checks stay clean
        prio = 0;
    }
    cudaStream_t s = nullptr;
    SEM_CU(ctx, cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio));
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaEventDestroy(ev[j]);
            cudaStreamDestroy(s);
            return sem_cuda(ctx, e, "cudaEventCreateWithFlags");
        }
    }
    ctx->aux = s;
    ctx->ev_fork = ev[0];
    ctx->ev_qseg = ev[1];
    ctx->ev_join = ev[2];
    return SEM_OK;
}

// the further fields' passes, on ctx->stream (whichever stream that is at the time); with
// `wait_q`, the first append waits for ev_qseg (Q's segment starts)
template <int NP>
static sem_status fields_passes(sem_ctx *ctx, const sem_mesh *m, int nf, const float *const *fields,
                                const IsoSet *SF, const IsoScratch *XF, float *tris, int32_t *tri_elem, int64_t cap,
                                int64_t *cd, bool wait_q, bool draw, int seg0)
{
    for (int k = 0; k < nf; ++k) {
        SEM_TRY(launch_count<NP>(ctx, fields[k], SF[k], m->E, XF[k].cnt, nullptr));
        SEM_TRY(iso_scan_async(ctx, m->E * SF[k].niso, XF[k]));
        if (k == 0 && wait_q) SEM_CU(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_qseg, 0));
        SEM_TRY(iso_segments_async(ctx, m->E, SF[k].niso, XF[k].offs, cd, true));
        if (tris) SEM_TRY(emit<NP>(ctx, m, fields[k], SF[k], XF[k].offs, XF[k].live, tris, tri_elem, cap, XF[k].next, cd));
        if (draw && tris) SEM_TRY(render_frame_draw(ctx, tris, seg0, seg0 + SF[k].niso, 1 + k));
        cd += SF[k].niso;
        seg0 += SF[k].niso;
    }
    return SEM_OK;
}

template <int NP>
static sem_status q_fields_np(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                              float *Q, const IsoSet &SQ, int nf, const float *const *fields, const IsoSet *SF,
                              float *tris, int32_t *tri_elem, int64_t cap, int64_t *counts_dev, bool draw)
{
    const int64_t E = m->E;
    IsoScratch XQ, XF[SEM_MAX_FIELDS];
    SEM_TRY(iso_scratch_async(ctx, E * SQ.niso, XQ, SCR_ISO));
    for (int k = 0; k < nf; ++k) SEM_TRY(iso_scratch_async(ctx, E * SF[k].niso, XF[k], SCR_ISO_F0 + k));
    // the Q kernel, counting Q's triangles itself where it can
    if (NP == 8 && !m->curved) {
        SEM_TRY(qcrit_count_launch(ctx, m, u, v, w, Q, SQ.niso, SQ.iso, XQ.cnt));
    } else {
        SEM_TRY(qcrit_launch(ctx, m, u, v, w, Q));
        SEM_TRY(launch_count<NP>(ctx, Q, SQ, E, XQ.cnt, nullptr));
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    // one stream while the kernel trace is on (each traced kernel's time is then its own) or an
    // emit launch is still to be timed (so are the tuner's timings), and under a capture that
    // began before the auxiliary stream existed (creating a stream is not done during capture)
    if (nf > 0 && cs == cudaStreamCaptureStatusNone) SEM_TRY(aux_ready(ctx));  // whether it forks or not
    bool fork = nf > 0 && !ctx->trace_on && ctx->aux;
    if (fork && cs == cudaStreamCaptureStatusNone && tris) {
        fork = emit_settled(ctx, m, SQ.niso);
        for (int k = 0; k < nf && fork; ++k) fork = emit_settled(ctx, m, SF[k].niso);
    }
    if (!fork) {
        SEM_TRY(iso_tail_async<NP>(ctx, m, Q, SQ, XQ, tris, tri_elem, cap, counts_dev, false));
        if (draw && tris) SEM_TRY(render_frame_draw(ctx, tris, 0, SQ.niso, 0));
        return fields_passes<NP>(ctx, m, nf, fields, SF, XF, tris, tri_elem, cap, counts_dev + SQ.niso, false, draw,
                                 SQ.niso);
    }
    SEM_TRY(aux_ready(ctx));
    cudaStream_t main = ctx->stream;
    SEM_CU(ctx, cudaEventRecord(ctx->ev_fork, main));
    SEM_CU(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    // Q's scan and segment starts, then the fields' passes on aux, then Q's emit; the join is
    // recorded whatever happens, so a capture in progress never holds an unjoined stream
    sem_status st = iso_scan_async(ctx, E * SQ.niso, XQ);
    if (st == SEM_OK) st = iso_segments_async(ctx, E, SQ.niso, XQ.offs, counts_dev, false);
    if (st == SEM_OK) st = sem_cuda(ctx, cudaEventRecord(ctx->ev_qseg, main), "cudaEventRecord");
    ctx->stream = ctx->aux;
    if (st == SEM_OK)
        st = fields_passes<NP>(ctx, m, nf, fields, SF, XF, tris, tri_elem, cap, counts_dev + SQ.niso, true, draw,
                               SQ.niso);
    ctx->stream = main;
    const cudaError_t ej = cudaEventRecord(ctx->ev_join, ctx->aux);
    if (st == SEM_OK && tris) st = emit<NP>(ctx, m, Q, SQ, XQ.offs, XQ.live, tris, tri_elem, cap, XQ.next);
    if (st == SEM_OK && draw && tris) st = render_frame_draw(ctx, tris, 0, SQ.niso, 0);
    const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(main, ctx->ev_join, 0) : ej;
    SEM_TRY(st);
    return sem_cuda(ctx, ew, "join of the auxiliary stream");
}

sem_status iso_run_q_fields_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                                  float *Q, const float *q_isos, int q_niso, int nf, const float *const *fields,
                                  const float *f_isos, const int *f_niso, float *tris, int32_t *tri_elem,
                                  int64_t cap, int64_t *counts_dev, bool draw)
{
    IsoSet SQ, SF[SEM_MAX_FIELDS];
    memset(&SQ, 0, sizeof SQ);
    memset(SF, 0, sizeof SF);
    SQ.niso = q_niso;
    for (int q = 0; q < q_niso; ++q) SQ.iso[q] = q_isos[q];
    for (int k = 0, at = 0; k < nf; ++k) {
        SF[k].niso = f_niso[k];
        for (int q = 0; q < f_niso[k]; ++q) SF[k].iso[q] = f_isos[at++];
    }
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return q_fields_np<NPV>(ctx, m, u, v, w, Q, SQ, nf, fields, SF, tris, tri_elem, cap, counts_dev, draw);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status iso_run_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso,
                               float *tris, int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases,
                               bool append)
{
    IsoSet S;
    memset(&S, 0, sizeof S);
    S.niso = niso;
    for (int q = 0; q < niso; ++q) S.iso[q] = isos[q];
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_multi_async_np<NPV>(ctx, m, f, S, tris, tri_elem, cap, counts_dev, cases, append);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status iso_run_multi(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso, float *tris,
                         int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    IsoSet S;
    memset(&S, 0, sizeof S);
    S.niso = niso;
    for (int q = 0; q < niso; ++q) S.iso[q] = isos[q];
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_multi_np<NPV>(ctx, m, f, S, tris, tri_elem, cap, ntri_out, cases);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status iso_run(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris, int32_t *tri_elem,
                   int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    return iso_run_multi(ctx, m, f, &iso, 1, tris, tri_elem, cap, ntri_out, cases);
}

// ==========================================================================================
// Allocation-free variant of sem_isosurface (sem_isosurface_noalloc).  Same kernels and the
// same scan; the per-element counts, offsets and scan partials live in one file-scope device
// array instead of the context's grow-only arena, so a call never allocates.
// ==========================================================================================
namespace {
constexpr size_t al256(size_t b) { return ((b + 255) / 256) * 256; }
constexpr int64_t kNaMaxE = SEM_NOALLOC_MAX_ELEMENTS;
constexpr size_t kNaCnt = al256(sizeof(int32_t) * kNaMaxE);
constexpr size_t kNaOff = al256(sizeof(int64_t) * (kNaMaxE + 1));
constexpr size_t kNaTmp = al256(sizeof(int64_t) * ((kNaMaxE + 4095) / 4096 + 1));
}  // namespace

// Shared by every call on a device; holds the last call's contents until the next call.
// Nothing in it needs to start at zero: every word is written before it is read.
static __device__ __align__(256) unsigned char g_iso_noalloc_scratch[kNaCnt + kNaOff + kNaTmp];

template <int NP>
static cudaError_t noalloc_load_kernels()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_iso_count<NP>);
    return e != cudaSuccess ? e : cudaFuncGetAttributes(&a, k_iso_emit<NP>);
}

// Set-up of sem_isosurface_noalloc for ctx->device (current), run by sem_create: the device
// address of g_iso_noalloc_scratch (in host code the symbol is only a stand-in), kept in the
// context, and the kernels the entry point launches, so that with lazy module loading neither
// the array nor any of its code is loaded -- which would allocate -- during a call.  Querying a
// kernel's attributes takes its handle, which makes the runtime load it.
sem_status iso_noalloc_prepare(sem_ctx *ctx)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_iso_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return sem_cuda(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    ctx->noalloc_scratch = p;
#define SEM_CASE(NPV) if ((e = noalloc_load_kernels<NPV>()) != cudaSuccess) return sem_cuda(ctx, e, "cudaFuncGetAttributes");
    SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
    SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    return scan_load_kernels(ctx);
}

template <int NP>
static sem_status iso_run_noalloc_np(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                                     int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    const int64_t E = m->E;
    if (scan_tmp_bytes(E) > kNaTmp) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_noalloc: scan scratch too small");
    char *scr = static_cast<char *>(ctx->noalloc_scratch);
    if (!scr) return sem_fail(ctx, SEM_ERR_CUDA, "sem_isosurface_noalloc: scratch address not resolved");
    int32_t *cnt = reinterpret_cast<int32_t *>(scr);
    int64_t *offs = reinterpret_cast<int64_t *>(scr + kNaCnt);
    void *tmp = scr + kNaCnt + kNaOff;
    constexpr int WV = IsoW<NP>::V;
    const unsigned grid = (unsigned)((E + WV - 1) / WV);
    SEM_TRACED(ctx, "k_iso_count", k_iso_count<NP><<<grid, 32 * WV, 0, ctx->stream>>>(f, iso, E, cnt, cases));
    SEM_CU(ctx, cudaGetLastError());
    SEM_TRY(scan_i32_i64(ctx, cnt, offs, E, tmp));
    SEM_CU(ctx, cudaMemcpyAsync(ctx->h_pinned, offs + E, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t total = ctx->h_pinned[0];
    *ntri_out = total;
    if (!tris) return SEM_OK;
    if (total > cap)
        return sem_fail(ctx, SEM_ERR_CAPACITY, "sem_isosurface_noalloc: %lld triangles exceed capacity %lld",
                        (long long)total, (long long)cap);
    if (total == 0) return SEM_OK;
    SEM_TRACED(ctx, "k_iso_emit", k_iso_emit<NP><<<grid, 32 * WV, 0, ctx->stream>>>(f, iso, E, offs, m->lo, m->hi, tris, tri_elem, cap));
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_emit launch");
}

sem_status iso_run_noalloc(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                           int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_run_noalloc_np<NPV>(ctx, m, f, iso, tris, tri_elem, cap, ntri_out, cases);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}
