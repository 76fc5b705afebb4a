// sem_qcrit_tc.cu -- Q-criterion with the s- and t-contractions on the tensor cores (tcgen05),
// in BF16, FP16, split BF16 (hi + lo) or TF32, FP32 accumulation; N = 7 elements.
//
// For one element component U (64 node rows (k, j) x 8 columns i) the two contractions are
//   S[(k,j), i] = sum_m D[j][m] U[(k,m), i],   T[(k,j), i] = sum_m D[k][m] U[(m,j), i],
// i.e. S = (I8 (x) D) U and T = (D (x) I8) U: one 128 x 64 constant matrix A = [I8(x)D ; D(x)I8]
// times U, and the element components of a tile batch along N.  A second MMA with the stacked
// A = [I8(x)D ; D(x)I8 ; I8(x)D] read from row 64 puts S and T in every TMEM lane quarter, so all
// eight warps find S and T of their node lines in their own lanes and run the Q epilogue; the
// r-contraction (K = 8) stays on FP32 FFMA from the FP32 copy of the element in shared memory.
// The element data is staged by the TMA engine (cp.async.bulk), converted to the operand type and
// transposed into the K-major 128-byte-swizzled operand layout by the CUDA cores.  A 16-bit row
// of K = 64 fills one 128-byte swizzle atom; a TF32 row fills two, stored as two K blocks (K 0-31
// and 32-63) each laid out like the 16-bit tile, and an MMA (32 bytes of K: 16 16-bit or 8 TF32
// values) never crosses from one block into the other.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <string.h>

#include <vector>

#include "sem_internal.cuh"
#include "sem_tc.cuh"

namespace {

constexpr int NP = 8, NP3 = 512;
constexpr int NE = 4;                 // elements per tile
constexpr int NS = 3 * NE;            // element components (slots) per tile
constexpr int NCOL = 8 * NS;          // MMA N = 96
constexpr int SLOT_F = 520;           // floats per staged slot (512 + 8 padding: conflict-free transpose)
constexpr int A_ROWS = 192;           // [I(x)D ; D(x)I ; I(x)D]
constexpr int STAGE_BYTES = NS * SLOT_F * 4;
// operand arithmetic of the s- and t-contractions
constexpr int P_FP16 = 0, P_BF16 = 1, P_BF16X2 = 2, P_TF32 = 3;
constexpr int TMEM_COLS = 512;
// warp roles: 0-7 epilogue (warp w reads TMEM lane quarter w % 4), 8-11 convert, 12 TMA, 13 MMA
constexpr int EPI_WARPS = 8, CVT_WARPS = 4;
constexpr int TMA_WARP = EPI_WARPS + CVT_WARPS, MMA_WARP = TMA_WARP + 1;
constexpr int THREADS = 32 * (MMA_WARP + 1);

template <int PREC>
struct Smem {
    static constexpr bool SPLIT = PREC == P_BF16X2, TF32 = PREC == P_TF32;
    static constexpr int KB = TF32 ? 2 : 1;               // K blocks of 128-byte rows
    static constexpr int A_BYTES = KB * A_ROWS * 128;
    static constexpr int B_BYTES = KB * NCOL * 128;
    static constexpr int NA = SPLIT ? 2 : 1;
    static constexpr int NSTAGE = (SPLIT || TF32) ? 4 : 5;  // TMA ring of FP32 element tiles
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = A_OFF + NA * A_BYTES;                 // 2 buffers x NA
    static constexpr int ST_OFF = B_OFF + 2 * NA * B_BYTES;
    static constexpr int BAR_OFF = ST_OFF + NSTAGE * STAGE_BYTES;
    // barriers: full[5] sfree[5] bready[2] bfree[2] accfull[2] accfree[2] abar -> 19
    static constexpr int TOTAL = BAR_OFF + 20 * 8 + 16;
    static constexpr int ALLOC = TOTAL + 1024;  // room to align the base to 1024 B
};

}  // namespace

__constant__ float c_Dtc[NP * NP];  // FP32 D for the r-contraction (N = 7)

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if constexpr (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

template <bool BF16>
__device__ __forceinline__ float round16(float a)
{
    if constexpr (BF16) return __bfloat162float(__float2bfloat16_rn(a));
    else return __half2float(__float2half_rn(a));
}

// FP32 -> TF32 (10 explicit mantissa bits), round to nearest with ties away from zero, in a
// 32-bit container whose low 13 bits are zero
__device__ __forceinline__ uint32_t to_tf32(float a)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// barrier over `nthreads` threads that also ORs a predicate across them (uniform result)
__device__ __forceinline__ bool named_sync_or(int id, int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Warp-specialised pipeline over tiles of NE elements:
//   producer (warp 12, lane 0): bulk-copies the u, v, w of a tile into a free ring stage;
//   converters (warps 8-11): 16-bit conversion + transpose of the stage into a free B buffer;
//   MMA issuer (warp 13, lane 0): 2 x 4 MMAs (x3 products when split) into a free TMEM set;
//   epilogue (warps 0-7): S and T from TMEM, r by FFMA from the stage, Q, 16-byte stores.
// Every hand-off is an mbarrier; every wait is bounded and raises the error flag on expiry.
template <int PREC>
__global__ void __launch_bounds__(THREADS, 1) k_sem_q_tc(const float *__restrict__ f0, const float *__restrict__ f1,
                                                         const float *__restrict__ f2, float *__restrict__ Q,
                                                         const float4 *__restrict__ gfac, int64_t E,
                                                         const uint8_t *__restrict__ A_glob, int *err)
{
    using L = Smem<PREC>;
    constexpr int NSTAGE = L::NSTAGE;
    constexpr bool SPLIT = L::SPLIT, TF32 = L::TF32, BF16 = PREC == P_BF16 || PREC == P_BF16X2;
    constexpr int A_BYTES = L::A_BYTES, B_BYTES = L::B_BYTES;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t *sA = sm + L::A_OFF;
    uint8_t *sB = sm + L::B_OFF;
    float *stage = reinterpret_cast<float *>(sm + L::ST_OFF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::BAR_OFF);
    uint64_t *full = bars, *sfree = bars + 5, *bready = bars + 10, *bfree = bars + 12, *accfull = bars + 14,
             *accfree = bars + 16, *abar = bars + 18;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 19);
    volatile int *s_abort = reinterpret_cast<volatile int *>(bars + 19) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (E + NE - 1) / NE;

    if (tid == 0) {
        *s_abort = 0;
        for (int b = 0; b < NSTAGE; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&sfree[b], 32 * EPI_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bready[b], 1);
            mbar_init(&bfree[b], 1);
            mbar_init(&accfull[b], 1);
            mbar_init(&accfree[b], 32 * EPI_WARPS);
        }
        mbar_init(abar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(s_tmem, TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;

    if (warp == TMA_WARP) {
        // ------------------------------------------------ producer: one thread keeps the ring full
        if (lane == 0) {
            const float *src[3] = {f0, f1, f2};
            mbar_arrive_expect_tx(abar, L::NA * A_BYTES);
            bulk_g2s(sA, A_glob, L::NA * A_BYTES, abar);
            int it_p = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it_p) {
                const int s = it_p % NSTAGE;
                if (!mbar_wait_bounded(&sfree[s], ((it_p / NSTAGE) & 1) ^ 1, err)) *s_abort = 1;
                if (*s_abort) break;
                const int64_t ne = (E - tile * NE) < NE ? (E - tile * NE) : NE;
                float *dst = stage + s * NS * SLOT_F;
                mbar_arrive_expect_tx(&full[s], (uint32_t)(ne * 3 * 2048));
                for (int e_l = 0; e_l < ne; ++e_l)
                    for (int c = 0; c < 3; ++c)
                        bulk_g2s(dst + (e_l * 3 + c) * SLOT_F, src[c] + (tile * NE + e_l) * NP3, 2048, &full[s]);
            }
            // on an abort, wait (bounded) for the copies still in flight into the ring
            if (*s_abort)
                for (int k = it_p > NSTAGE ? it_p - NSTAGE : 0; k < it_p; ++k)
                    mbar_wait_bounded(&full[k % NSTAGE], (k / NSTAGE) & 1, nullptr);
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------ MMA issuer: one thread
        if (lane == 0) {
            constexpr uint32_t IDESC = TF32 ? tc::idesc_tf32(128, NCOL) : tc::idesc_f16(128, NCOL, BF16);
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            if (!mbar_wait_bounded(abar, 0, err)) *s_abort = 1;
            int it_m = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it_m) {
                const int b = it_m & 1, t = it_m & 1;
                const uint32_t pb = (it_m >> 1) & 1;
                if (!mbar_wait_bounded(&bready[b], pb, err)) *s_abort = 1;
                if (!mbar_wait_bounded(&accfree[t], pb ^ 1, err)) *s_abort = 1;
                if (*s_abort) break;
                tc::fence_after_sync();
                const uint32_t bb0 = b0 + b * L::NA * B_BYTES;
                for (int half = 0; half < 2; ++half) {
                    const uint32_t d = tmem + t * 2 * NCOL + half * NCOL;
                    const uint32_t aoff = half * 64 * 128;  // A rows 64.. within each K block
                    int acc = 0;
                    const int nterm = SPLIT ? 3 : 1;
                    for (int term = 0; term < nterm; ++term) {
                        // split: hi*hi, hi*lo (B lo), lo*hi (A lo)
                        const uint32_t aa = a0 + aoff + (term == 2 ? A_BYTES : 0);
                        const uint32_t bb = bb0 + (term == 1 ? B_BYTES : 0);
                        // 32 bytes of K per MMA; K block kk / 4 of the operands
                        for (int kk = 0; kk < 4 * L::KB; ++kk) {
                            const uint32_t ka = (kk >> 2) * (A_ROWS * 128) + (kk & 3) * 32;
                            const uint32_t kb = (kk >> 2) * (NCOL * 128) + (kk & 3) * 32;
                            if constexpr (TF32)
                                tc::mma_tf32(d, tc::desc_k_sw128(aa + ka), tc::desc_k_sw128(bb + kb), IDESC, acc);
                            else
                                tc::mma_f16(d, tc::desc_k_sw128(aa + ka), tc::desc_k_sw128(bb + kb), IDESC, acc);
                            acc = 1;
                        }
                    }
                }
                tc::commit(&accfull[t]);
                tc::commit(&bfree[b]);
            }
        }
    } else if (warp >= EPI_WARPS) {
        // ------------------------------------------------ converters (128 threads)
        const int ct = tid - 32 * EPI_WARPS;
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % NSTAGE, b = it & 1;
            bool bad = !mbar_wait_bounded(&full[s], (it / NSTAGE) & 1, err);
            bad = bad || !mbar_wait_bounded(&bfree[b], ((it >> 1) & 1) ^ 1, err);
            bad = bad || *s_abort;
            // all converter threads take the same decision (they meet at a named barrier below)
            if (named_sync_or(2, 32 * CVT_WARPS, bad)) {
                *s_abort = 1;
                break;
            }
            const int64_t ne = (E - tile * NE) < NE ? (E - tile * NE) : NE;
            if (ct < NS * 8) {
                const int slot = ct >> 3, i = ct & 7;
                const bool live = slot / 3 < ne;
                const float *col = stage + s * NS * SLOT_F + slot * SLOT_F + i;
                uint8_t *rowB = sB + b * L::NA * B_BYTES + slot * 1024 + i * 128;
                // the column's level shift: (I (x) D) and (D (x) I) have rows summing to zero, so
                // subtracting the column's first value leaves S and T unchanged in exact arithmetic
                // and leaves only the column's variation to be rounded to the operand type
                const float c0 = live ? col[0] : 0.f;
#pragma unroll
                for (int kc = 0; kc < 8; ++kc) {
                    float v[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) v[t] = live ? col[(kc * 8 + t) * 8] - c0 : 0.f;
                    if constexpr (TF32) {
                        // K = 8 kc + t: block kc / 4, 16-byte chunks 2 (kc % 4) and 2 (kc % 4) + 1
                        uint8_t *rb = rowB + (kc >> 2) * (NCOL * 128);
                        const int c0 = 2 * (kc & 3);
                        *reinterpret_cast<uint4 *>(rb + ((c0 ^ i) * 16)) =
                            make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
                        *reinterpret_cast<uint4 *>(rb + (((c0 + 1) ^ i) * 16)) =
                            make_uint4(to_tf32(v[4]), to_tf32(v[5]), to_tf32(v[6]), to_tf32(v[7]));
                        continue;
                    }
                    uint4 hi;
                    hi.x = pack2<BF16>(v[0], v[1]);
                    hi.y = pack2<BF16>(v[2], v[3]);
                    hi.z = pack2<BF16>(v[4], v[5]);
                    hi.w = pack2<BF16>(v[6], v[7]);
                    *reinterpret_cast<uint4 *>(rowB + ((kc ^ i) * 16)) = hi;
                    if constexpr (SPLIT) {
                        uint4 lo;
                        lo.x = pack2<BF16>(v[0] - round16<BF16>(v[0]), v[1] - round16<BF16>(v[1]));
                        lo.y = pack2<BF16>(v[2] - round16<BF16>(v[2]), v[3] - round16<BF16>(v[3]));
                        lo.z = pack2<BF16>(v[4] - round16<BF16>(v[4]), v[5] - round16<BF16>(v[5]));
                        lo.w = pack2<BF16>(v[6] - round16<BF16>(v[6]), v[7] - round16<BF16>(v[7]));
                        *reinterpret_cast<uint4 *>(rowB + B_BYTES + ((kc ^ i) * 16)) = lo;
                    }
                }
            }
            tc::fence_proxy_async();
            named_sync(1, 32 * CVT_WARPS);
            if (ct == 0) mbar_arrive(&bready[b]);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0-7, TMEM quarter = warp % 4)
        const int q = warp & 3, lg = q & 1, hq = q >> 1;
        const int el = hq + 2 * (warp >> 2);  // quarters 0,1 -> elements 0,2; quarters 2,3 -> 1,3
        const int line = 32 * lg + lane;
        const int sw = (lane >> 2) & 1;       // row-chunk stagger: lines l and l+4 hit other banks
        const uint32_t t_lane = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t colS = hq ? NCOL : 0, colT = hq ? 0 : NCOL;
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % NSTAGE, t = it & 1;
            const int64_t e = tile * NE + el;
            const float4 g = gfac[e < E ? e : E - 1];
            if (!mbar_wait_bounded(&accfull[t], (it >> 1) & 1, err)) *s_abort = 1;
            if (!mbar_wait_bounded(&full[s], (it / NSTAGE) & 1, err)) *s_abort = 1;
            tc::fence_after_sync();
            const float *st = stage + s * NS * SLOT_F;
            {
                uint32_t rs[3][8], rt[3][8];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int slot = el * 3 + c;
                    tc::tmem_ld8(t_lane + t * 2 * NCOL + colS + slot * 8, rs[c]);
                    tc::tmem_ld8(t_lane + t * 2 * NCOL + colT + slot * 8, rt[c]);
                }
                // r-contraction from the FP32 rows while the TMEM loads are in flight
                float dr[3][8];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 *rp = reinterpret_cast<const float4 *>(st + (el * 3 + c) * SLOT_F + line * 8);
                    const float4 A = rp[sw], B = rp[sw ^ 1];
                    const float4 lo = sw ? B : A, hi = sw ? A : B;
                    // the row shifted by its first value (D's rows sum to zero): the rounding
                    // follows the variation along the row, not the values' magnitude
                    const float row[8] = {0.f, lo.y - lo.x, lo.z - lo.x, lo.w - lo.x,
                                          hi.x - lo.x, hi.y - lo.x, hi.z - lo.x, hi.w - lo.x};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float a = 0.f;
#pragma unroll
                        for (int m = 1; m < 8; ++m) a = fmaf(c_Dtc[i * 8 + m], row[m], a);
                        dr[c][i] = a;
                    }
                }
                tc::tmem_wait_ld();
                if (e < E && !*s_abort) {
                    const float c11 = -0.5f * g.x * g.x, c22 = -0.5f * g.y * g.y, c33 = -0.5f * g.z * g.z;
                    const float c12 = -g.x * g.y, c13 = -g.x * g.z, c23 = -g.y * g.z;
                    float qv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float us = __uint_as_float(rs[0][i]), ut = __uint_as_float(rt[0][i]);
                        const float vs = __uint_as_float(rs[1][i]), vt = __uint_as_float(rt[1][i]);
                        const float ws = __uint_as_float(rs[2][i]), wt = __uint_as_float(rt[2][i]);
                        float a = c11 * dr[0][i] * dr[0][i];
                        a = fmaf(c12 * us, dr[1][i], a);
                        a = fmaf(c22 * vs, vs, a);
                        a = fmaf(c13 * ut, dr[2][i], a);
                        a = fmaf(c23 * vt, ws, a);
                        a = fmaf(c33 * wt, wt, a);
                        qv[i] = a;
                    }
                    float4 *dst = reinterpret_cast<float4 *>(Q + e * NP3 + line * 8);
                    dst[0] = make_float4(qv[0], qv[1], qv[2], qv[3]);
                    dst[1] = make_float4(qv[4], qv[5], qv[6], qv[7]);
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&accfree[t]);
            mbar_arrive(&sfree[s]);
            // warp-uniform exit: tcgen05.ld is a whole-warp instruction
            if (__any_sync(0xffffffffu, *s_abort != 0)) break;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------ host

// Nearest TF32 (10 explicit mantissa bits, ties to even) of a finite float, in a 32-bit container
static float host_tf32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= ~0x1FFFu;
    memcpy(&x, &u, 4);
    return x;
}

// A stack [I(x)D ; D(x)I ; I(x)D] in the swizzled K-major layout, for N = 7:
// A_S[(k,j),(k',m)] = d(k,k') D[j][m];  A_T[(k,j),(m,j')] = D[k][m] d(j,j').
// 16-bit (bf16 or fp16, hi and the lo remainder) or TF32 (two K blocks, out_lo unused).
static void build_A(const double *D, int prec, std::vector<uint8_t> &out_hi, std::vector<uint8_t> &out_lo)
{
    const bool tf32 = prec == P_TF32, bf16 = prec == P_BF16 || prec == P_BF16X2;
    const size_t bytes = (size_t)(tf32 ? 2 : 1) * A_ROWS * 128;
    out_hi.assign(bytes, 0);
    out_lo.assign(bytes, 0);
    for (int r = 0; r < A_ROWS; ++r) {
        const int rr = r % 128, part = (r < 64 || r >= 128) ? 0 : 1;  // 0: S rows, 1: T rows
        const int k = (rr % 64) / 8, j = (rr % 64) % 8;
        for (int kc = 0; kc < 64; ++kc) {
            const int a = kc / 8, b = kc % 8;  // node row (a, b)
            double v = 0.0;
            if (part == 0) v = (a == k) ? D[j * 8 + b] : 0.0;
            else v = (b == j) ? D[k * 8 + a] : 0.0;
            if (tf32) {
                const int blk = kc / 32, e = kc % 32;
                const size_t off = (size_t)blk * A_ROWS * 128 + (size_t)(r / 8) * 1024 + (r % 8) * 128 +
                                   (((e / 4) ^ (r % 8)) * 16) + (e % 4) * 4;
                const float t = host_tf32((float)v);
                memcpy(&out_hi[off], &t, 4);
                continue;
            }
            const size_t off = (size_t)(r / 8) * 1024 + (r % 8) * 128 + (((kc / 8) ^ (r % 8)) * 16) + (kc % 8) * 2;
            uint16_t h, l;
            if (bf16) {
                __nv_bfloat16 hh = __double2bfloat16(v);
                __nv_bfloat16 ll = __double2bfloat16(v - (double)__bfloat162float(hh));
                memcpy(&h, &hh, 2);
                memcpy(&l, &ll, 2);
            } else {
                __half hh = __double2half(v);
                __half ll = __double2half(v - (double)__half2float(hh));
                memcpy(&h, &hh, 2);
                memcpy(&l, &ll, 2);
            }
            memcpy(&out_hi[off], &h, 2);
            memcpy(&out_lo[off], &l, 2);
        }
    }
}

template <int PREC>
static sem_status launch_tc(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q,
                            const uint8_t *A)
{
    using L = Smem<PREC>;
    static_assert(L::ALLOC <= 232448, "shared memory per CTA");
    auto kern = k_sem_q_tc<PREC>;
    static KernelSetup ks;  // per instantiation and device
    SEM_TRY(kernel_setup(ctx, ks, kern, 0, L::ALLOC));
    // one CTA per SM: it allocates all 512 TMEM columns (two accumulator sets)
    const int64_t ntiles = (m->E + NE - 1) / NE;
    int64_t grid = (int64_t)ctx->sm_count;
    if (grid > ntiles) grid = ntiles;
    SEM_TRACED(ctx, "k_sem_q_tc", kern<<<(unsigned)grid, THREADS, L::ALLOC, ctx->stream>>>(u, v, w, Q, m->g, m->E, A, ctx->d_flag));
    return sem_cuda(ctx, cudaGetLastError(), "k_sem_q_tc launch");
}

sem_status qcrit_tc_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q,
                           sem_prec prec, const double *D64)
{
    if (m->N != 7)
        return sem_fail(ctx, SEM_ERR_UNSUPPORTED, "tensor-core precisions are built for N = 7 only (N=%d)", m->N);
    // operand tables: 0 bf16 (hi + lo), 1 fp16 (hi + lo), 2 tf32
    const int slot = prec == SEM_FP16 ? 1 : (prec == SEM_TF32 ? 2 : 0);
    const int tprec = slot == 0 ? P_BF16 : (slot == 1 ? P_FP16 : P_TF32);
    if (!ctx->tc_A[slot]) {
        std::vector<uint8_t> hi, lo;
        build_A(D64, tprec, hi, lo);
        std::vector<uint8_t> both(hi);
        both.insert(both.end(), lo.begin(), lo.end());
        void *d = nullptr;
        SEM_CU(ctx, cudaMalloc(&d, both.size()));
        ctx->mem_add((int64_t)both.size());
        SEM_CU(ctx, cudaMemcpy(d, both.data(), both.size(), cudaMemcpyHostToDevice));
        ctx->tc_A[slot] = d;
        float Df[64];
        for (int q = 0; q < 64; ++q) Df[q] = (float)D64[q];
        SEM_CU(ctx, cudaMemcpyToSymbol(c_Dtc, Df, sizeof Df));
    }
    const uint8_t *A = static_cast<const uint8_t *>(ctx->tc_A[slot]);
    switch (prec) {
    case SEM_BF16: return launch_tc<P_BF16>(ctx, m, u, v, w, Q, A);
    case SEM_FP16: return launch_tc<P_FP16>(ctx, m, u, v, w, Q, A);
    case SEM_BF16X2: return launch_tc<P_BF16X2>(ctx, m, u, v, w, Q, A);
    case SEM_TF32: return launch_tc<P_TF32>(ctx, m, u, v, w, Q, A);
    default: return sem_fail(ctx, SEM_ERR_UNSUPPORTED, "precision %d has no tensor-core kernel", (int)prec);
    }
}
