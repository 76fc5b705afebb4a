// sem_ae.cu -- the learned per-element compression: an MLP autoencoder trained and run on the
// 5th-generation tensor cores in BF16 with FP32 accumulation.
//
// Method (the per-element compression for in-transit transfer, Sec. 4.2's motivation): per
// element of order N = 7 the 3 x 512 nodal velocity values, z-scored per component, go
// through
//     encoder  H1 = X W1^T + b1, A1 = gelu(H1), Z = A1 W2^T + b2     (1536 -> 512 -> 48)
//     decoder  H3 = Z W3^T + b3, A3 = gelu(H3), Y = A3 W4^T + b4     (48 -> 512 -> 1536)
// gelu(x) = x Phi(x) (exact, via erff), loss = mean (Y - X)^2, AdamW updates (Loshchilov &
// Hutter 2019).  The latent Z is stored in BF16: the decoder and the training graph both see
// the BF16 latent, whose gradient passes through the rounding unchanged.
//
// Design (GB300): every product is one tcgen05 GEMM D[M][N] = A[M][K] B[N][K]^T with both
// operands K-major BF16 tiles brought into shared memory by TMA (2-D tensor maps, 128-byte
// swizzle), the accumulator in TMEM (128 lanes x BN FP32 columns), one elected thread issuing
// the MMAs, and four epilogue warps reading TMEM back and applying the layer's fused tail
// (bias, gelu, gelu', loss and its gradient, de-normalisation) before storing.  Products that
// need a transposed operand (dW = dH^T A) take a transposed copy that the producing epilogue
// wrote alongside the row-major one, so no GEMM needs an MN-major operand.  Widths are padded
// to multiples of 64 (the 48-wide latent to 64 with zero weights, which stay zero).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sem_internal.cuh"
#include "sem_tc.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int BM = 128, BK = 64, GEMM_THREADS = 192;

enum EpiMode : int {
    EPI_F32 = 0,        // C32 = acc                                    (weight gradients)
    EPI_BIAS_GELU = 1,  // H = acc + b -> out (H), aux (gelu H), out_t (gelu H)^T
    EPI_BIAS = 2,       // Z = acc + b -> out, out_t                     (latent)
    EPI_LOSS = 3,       // Y = acc + b; R = Y - X -> out (dY = scale R), out_t, loss += R^2
    EPI_DGELU = 4,      // dH = acc * gelu'(H_in) -> out, out_t
    EPI_PLAIN = 5,      // acc -> out, out_t
    EPI_DECODE = 6,     // Y = acc + b -> fields[c][row][node] = Y std_c + mean_c
    EPI_LATENT = 7,     // Z = acc + b -> out[row][0..47] (the transmitted latent)
};

struct EpiArgs {
    int mode;
    int64_t m_valid;     // rows >= m_valid are padding: nothing is stored for them
    const float *bias;   // [N]
    bf16 *out;           // row-major, leading dimension ld_out
    int ld_out;
    bf16 *out_t;         // transposed [N][ld_t]
    int ld_t;
    bf16 *aux;           // EPI_BIAS_GELU: gelu(H), leading dimension ld_out
    const bf16 *in;      // EPI_DGELU: H; EPI_LOSS: target X (leading dimension ld_in)
    int ld_in;
    float *c32;          // EPI_F32, leading dimension ld_out
    int64_t split_stride;  // EPI_F32 with a split K range: floats between the partial arrays
    float *loss;         // EPI_LOSS accumulator
    float scale;         // EPI_LOSS: 2 / (B D)
    float *fields[3];    // EPI_DECODE
    float mean[3], stdv[3];
    int np3;
};

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void store8_bf16(bf16 *p, const float (&v)[8])
{
    __align__(16) bf16 t[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) t[c] = __float2bfloat16_rn(v[c]);
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(t);
}

__device__ __forceinline__ void load8_bf16(const bf16 *p, float (&v)[8])
{
    const uint4 raw = *reinterpret_cast<const uint4 *>(p);
    const bf16 *t = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __bfloat162float(t[c]);
}

// The transposed copy (out_t) of the warp's 32 rows goes through shared memory: element (column
// c, row lane) at tstage[c * 32 + lane], written back after the warp's last column as 16-byte
// chunks of 8 rows, so a store covers 8 columns x 64 bytes instead of one 2-byte value per column.
__device__ __forceinline__ void put_t(bf16 *__restrict__ tstage, int cl, float x)
{
    tstage[cl * 32 + (threadIdx.x & 31)] = __float2bfloat16_rn(x);
}

// Modes whose row-major BF16 output (and input) goes through the warp's staged row segments:
// the lanes hold one row each, so direct 16-byte accesses would touch 32 rows per instruction;
// staged, each 64-byte row segment of a 32-column round is read or written by 4 lanes at once.
__device__ __forceinline__ bool staged_rows(int mode)
{
    return mode == EPI_BIAS_GELU || mode == EPI_BIAS || mode == EPI_PLAIN || mode == EPI_LOSS || mode == EPI_DGELU;
}

// The fused tail of one row's 8 consecutive output columns n .. n+7 (cl: n's column in the tile).
// For the staged modes, sr / sr2 are the lane's 8 columns in the round's staged rows: the input
// (EPI_LOSS's target, EPI_DGELU's H) is read from sr and the output (EPI_BIAS_GELU: H to sr,
// gelu H to sr2) written there, for the warp to store.
__device__ __forceinline__ void epilogue8(const EpiArgs &P, int64_t row, int n, int cl, float (&v)[8],
                                          float &loss_acc, float *__restrict__ c32, bf16 *__restrict__ tstage,
                                          bf16 *__restrict__ sr, bf16 *__restrict__ sr2)
{
    if (row >= P.m_valid) {
        if (P.mode == EPI_LOSS) {
            // padding rows of a partial batch carry no gradient (their stale values would
            // otherwise reach the weight gradients)
            const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            store8_bf16(sr, z);
        }
        // the transposed copy's padding rows are zero in every mode (the staging tile is written
        // back whole)
        if (P.out_t)
#pragma unroll
            for (int c = 0; c < 8; ++c) put_t(tstage, cl + c, 0.f);
        return;
    }
    switch (P.mode) {
    case EPI_F32: {
        float4 *dst = reinterpret_cast<float4 *>(c32 + row * P.ld_out + n);
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        return;
    }
    case EPI_BIAS_GELU: {
        float a[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            v[c] += P.bias[n + c];
            // gelu of the BF16-rounded pre-activation, the value the backward pass sees
            a[c] = gelu_f(__bfloat162float(__float2bfloat16_rn(v[c])));
        }
        store8_bf16(sr, v);
        store8_bf16(sr2, a);
#pragma unroll
        for (int c = 0; c < 8; ++c) put_t(tstage, cl + c, a[c]);
        return;
    }
    case EPI_BIAS:
    case EPI_PLAIN: {
        if (P.mode == EPI_BIAS)
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] += P.bias[n + c];
        store8_bf16(sr, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) put_t(tstage, cl + c, v[c]);
        return;
    }
    case EPI_LOSS: {
        float x[8];
        load8_bf16(sr, x);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float r = v[c] + P.bias[n + c] - x[c];
            loss_acc = fmaf(r, r, loss_acc);
            v[c] = P.scale * r;
        }
        store8_bf16(sr, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) put_t(tstage, cl + c, v[c]);
        return;
    }
    case EPI_DGELU: {
        float h[8];
        load8_bf16(sr, h);
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] *= gelu_grad_f(h[c]);
        store8_bf16(sr, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) put_t(tstage, cl + c, v[c]);
        return;
    }
    case EPI_DECODE: {
        const int comp = n / P.np3, node = n % P.np3;
        float4 *dst = reinterpret_cast<float4 *>(P.fields[comp] + row * P.np3 + node);
        float y[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) y[c] = fmaf(v[c] + P.bias[n + c], P.stdv[comp], P.mean[comp]);
        dst[0] = make_float4(y[0], y[1], y[2], y[3]);
        dst[1] = make_float4(y[4], y[5], y[6], y[7]);
        return;
    }
    case EPI_LATENT: {
        if (n >= 48) return;
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] += P.bias[n + c];
        store8_bf16(P.out + row * 48 + n, v);
        return;
    }
    default: return;
    }
}

// The epilogue of one accumulator tile by epilogue warp q (TMEM lane quarter q: a warp may only
// read its own): TMEM 32 columns per round (four loads in flight, one wait), the fused tail of
// every 8 columns, the row-major BF16 traffic through the warp's staged row segments `rs` (two
// sets of 32 rows x EPI_RS, the second for EPI_BIAS_GELU's gelu H) and the transposed copy through
// its staging tile `tstage` (BN columns x 32 rows).  mt, nt: the tile's M and N indices; kz: its
// K slice (EPI_F32 with a split K range).
#define EPI_RS 40
template <int BN>
__device__ __forceinline__ void epilogue_tile(const EpiArgs &P, uint32_t tacc, int64_t mt, int nt, int kz, int q,
                                              int lane, bf16 *__restrict__ tstage, bf16 *__restrict__ rs)
{
    const int cbeg = 0, cend = BN;
    const int64_t row = mt * BM + q * 32 + lane;
    float loss_acc = 0.f;
    float *c32 = P.c32 + (int64_t)kz * P.split_stride;  // this K slice's partial array
    bf16 *rs2 = rs + 32 * EPI_RS;
    const bool staged = staged_rows(P.mode), stage_in = P.mode == EPI_LOSS || P.mode == EPI_DGELU;
    const int64_t row0 = mt * BM + q * 32;
    const int lr = lane >> 2, part = lane & 3;  // the warp's accesses: rows lr + 8 i, 16-byte part
    // 32 columns per TMEM round: four loads in flight, one wait
    for (int c0 = cbeg; c0 < cend; c0 += 32) {
        uint32_t r[4][8];
#pragma unroll
        for (int h = 0; h < 4; ++h) tc::tmem_ld8(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(c0 + 8 * h), r[h]);
        const int n0 = nt * BN + c0;
        if (stage_in) {
            // the round's input rows, 4 lanes per 64-byte row segment (padding rows: zero)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = lr + 8 * i;
                const int64_t g = row0 + rr;
                const uint4 x = g < P.m_valid ? *reinterpret_cast<const uint4 *>(P.in + g * P.ld_in + n0 + part * 8)
                                              : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(rs + rr * EPI_RS + part * 8) = x;
            }
            __syncwarp();
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[h][c]);
            epilogue8(P, row, n0 + 8 * h, c0 + 8 * h, v, loss_acc, c32, tstage, rs + lane * EPI_RS + 8 * h,
                      rs2 + lane * EPI_RS + 8 * h);
        }
        if (staged) {
            // the round's output rows, 4 lanes per 64-byte row segment; padding rows are
            // not stored, except EPI_LOSS's zero gradient
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = lr + 8 * i;
                const int64_t g = row0 + rr;
                if (g < P.m_valid || P.mode == EPI_LOSS) {
                    *reinterpret_cast<uint4 *>(P.out + g * P.ld_out + n0 + part * 8) =
                        *reinterpret_cast<const uint4 *>(rs + rr * EPI_RS + part * 8);
                    if (P.mode == EPI_BIAS_GELU)
                        *reinterpret_cast<uint4 *>(P.aux + g * P.ld_out + n0 + part * 8) =
                            *reinterpret_cast<const uint4 *>(rs2 + rr * EPI_RS + part * 8);
                }
            }
            __syncwarp();  // the staged rows are free for the next round
        }
    }
    const bool has_t = P.out_t && (P.mode == EPI_BIAS_GELU || P.mode == EPI_BIAS || P.mode == EPI_LOSS ||
                                   P.mode == EPI_DGELU || P.mode == EPI_PLAIN);
    if (has_t) {
        // out_t[n][row0 .. row0 + 31] for the tile's columns n: lane l takes column c + l / 4,
        // rows 8 (l % 4) .. + 7 (row0 and ld_t are multiples of 32, so 16-byte aligned)
        __syncwarp();
        const int cq = lane >> 2;
        for (int c = cbeg; c < cend; c += 8) {
            const int cl = c + cq;
            const uint4 val = *reinterpret_cast<const uint4 *>(tstage + cl * 32 + part * 8);
            *reinterpret_cast<uint4 *>(P.out_t + (int64_t)(nt * BN + cl) * P.ld_t + row0 + part * 8) = val;
        }
    }
    if (P.mode == EPI_LOSS) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, d);
        if (lane == 0) atomicAdd(P.loss, loss_acc);
    }
}

// D[M][N] = A[M][K] B[N][K]^T for one BM x BN output tile per CTA.  Warp 0: TMA producer;
// warp 1: TMEM owner and MMA issuer; warps 2..5: epilogue (warp w reads TMEM lanes
// 32 (w % 4) .. + 31).  NST-deep ring of (A, B) K-slices of BK = 64 BF16 (one 128-byte
// swizzle atom row).  Every wait is bounded: on a time-out the kernel records SEM_ERR_TIMEOUT,
// stops issuing, waits (bounded) for its copies in flight, frees TMEM and returns.
template <int BN, int NST>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K,
                const __grid_constant__ EpiArgs P, int *err)
{
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[NST], empty[NST], accf;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ int s_consumed[NST];
    // SW128 tiles need 1024-byte alignment
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's K slice (all of K unless split)
    const int nk_all = K / BK;
    const int kb0 = (int)((int64_t)blockIdx.z * nk_all / gridDim.z);
    const int nk = (int)((int64_t)(blockIdx.z + 1) * nk_all / gridDim.z) - kb0;
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            s_consumed[s] = 0;
        }
        mbar_init(&accf, 1);
        fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, BN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    int issued[NST] = {};
    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NST, round = kb / NST;
            if (round > 0 && !mbar_wait_bounded(&empty[s], (round - 1) & 1, err)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int *)&s_abort) break;
            uint8_t *a = smem + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(a, &tmA, (kb0 + kb) * BK, blockIdx.x * BM, &full[s]);
            tma_load_2d(a + A_BYTES, &tmB, (kb0 + kb) * BK, blockIdx.y * BN, &full[s]);
            ++issued[s];
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t IDESC = tc::idesc_f16(BM, BN, true);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NST, round = kb / NST;
            if (*(volatile int *)&s_abort || !mbar_wait_bounded(&full[s], round & 1, err)) {
                s_abort = 1;
                break;
            }
            s_consumed[s] = round + 1;
            tc::fence_after_sync();
            const uint32_t a = smem_u32(smem + s * STAGE_BYTES), b = a + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                tc::mma_f16(tmem, tc::desc_k_sw128(a + kk * 32), tc::desc_k_sw128(b + kk * 32), IDESC,
                            (kb | kk) != 0 ? 1u : 0u);
            tc::commit(&empty[s]);
        }
        tc::commit(&accf);  // also on an abort: the epilogue's wait then covers the issued MMAs
    } else if (warp >= 2) {
        // warp-uniform: the TMEM loads below are collective over the warp
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf, 0, err));
        if (!ok) s_abort = 1;
        tc::fence_after_sync();
        if (ok && !*(volatile int *)&s_abort) {
            // warps 2..5: one per TMEM lane quarter q = warp % 4.  The pipeline's shared memory is
            // idle once the accumulator is complete: warp q's staging tile and row segments live
            // there.
            const int q = warp & 3;
            bf16 *tstage = reinterpret_cast<bf16 *>(smem) + q * (BN * 32);
            bf16 *rs = reinterpret_cast<bf16 *>(smem) + 4 * (BN * 32) + q * (2 * 32 * EPI_RS);
            epilogue_tile<BN>(P, tmem, blockIdx.x, blockIdx.y, blockIdx.z, q, lane, tstage, rs);
        }
    }
    // on an abort: wait (bounded) for this CTA's copies still in flight
    if (warp == 0 && lane == 0 && *(volatile int *)&s_abort) {
        for (int s = 0; s < NST; ++s)
            if (issued[s] > s_consumed[s]) mbar_wait_bounded(&full[s], s_consumed[s] & 1, nullptr);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, BN);
    }
}

// ------------------------------------------------------------------------------------------
// element-wise kernels
// ------------------------------------------------------------------------------------------

// X[r][c] = (sample(r)[c] - mean) / std (BF16), and X^T; rows >= B are zero.  A sample is
// either row idx[r] of samples[n][3*np3] or element e0 + r of the fields u, v, w.  One block
// per 32 x 32 tile (rows r0.., columns c0..), transposed through shared memory so both X and
// X^T are written with coalesced stores.
__global__ void __launch_bounds__(256) k_pack(const float *__restrict__ samples, const int64_t *__restrict__ idx,
                                              int64_t n_samples, const float *__restrict__ f0,
                                              const float *__restrict__ f1, const float *__restrict__ f2, int64_t e0,
                                              int B, int Bp, int np3, float m0, float m1, float m2, float r0,
                                              float r1, float r2, bf16 *__restrict__ X, bf16 *__restrict__ XT,
                                              int *err)
{
    __shared__ bf16 tile[32][34];
    const int D = 3 * np3;
    const int c0 = blockIdx.x * 32, rbase = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int c = c0 + tx, comp = c / np3, node = c % np3;
    const float mean = comp == 0 ? m0 : comp == 1 ? m1 : m2, rs = comp == 0 ? r0 : comp == 1 ? r1 : r2;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = rbase + rr;
        float x = 0.f;
        if (r < B) {
            float raw = 0.f;
            if (samples) {
                const int64_t j = idx[r];
                if (j >= 0 && j < n_samples) {
                    raw = samples[j * D + c];
                } else {
                    // an index outside the sample array: flagged, and read as the mean
                    if (err) atomicOr(err, 1 << SEM_ERR_ARG);
                    raw = mean;
                }
            } else {
                raw = (comp == 0 ? f0 : comp == 1 ? f1 : f2)[(e0 + r) * np3 + node];
            }
            x = (raw - mean) * rs;
        }
        const bf16 b = __float2bfloat16_rn(x);
        X[(int64_t)r * D + c] = b;
        tile[rr][tx] = b;
    }
    if (!XT) return;
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) XT[(int64_t)(c0 + cc) * Bp + rbase + tx] = tile[tx][cc];
}

// latent [E][48] (BF16) rows e0 .. e0 + B - 1 -> Z [Bp][64] with zero padding
__global__ void k_latent_in(const bf16 *__restrict__ lat, int64_t e0, int B, int Bp, bf16 *__restrict__ Z)
{
    const int64_t total = (int64_t)Bp * 64;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / 64), c = (int)(t % 64);
        Z[t] = (r < B && c < 48) ? lat[(e0 + r) * 48 + c] : __float2bfloat16_rn(0.f);
    }
}

// out[n] = sum_{r < B} M^T[n][r]: one warp per row of a transposed BF16 matrix [N][ld]
// (16-byte loads, fixed summation order, so the result is deterministic)
__global__ void k_rowsum(const bf16 *__restrict__ MT, int N, int B, int ld, float *__restrict__ out)
{
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    const bf16 *row = MT + (int64_t)n * ld;
    float s = 0.f;
    const int B8 = B & ~7;
    for (int r = lane * 8; r < B8; r += 256) {
        float v[8];
        load8_bf16(row + r, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) s += v[c];
    }
    for (int r = B8 + lane; r < B; r += 32) s += __bfloat162float(row[r]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) out[n] = s;
}

struct TensorDesc {
    int64_t off;      // offset of the tensor in the flat FP32 arrays
    int rows, cols;   // padded shape (rows x cols), row-major
    int64_t wb_off;   // BF16 copy [rows][cols], -1 if none (biases)
    int64_t wt_off;   // BF16 transpose [cols][rows], -1 if none
};
constexpr int NT = 8;
struct AdamTable {
    TensorDesc t[NT];
};

// AdamW over every parameter (FP32 master, moments m and v), then the BF16 copies the GEMMs
// read: W [rows][cols] and W^T [cols][rows].
__global__ void k_adamw(const __grid_constant__ AdamTable T, int64_t n_total, float *__restrict__ w,
                        float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g, float lr, float b1,
                        float b2, float eps, float wd, float bc1, float bc2, bf16 *__restrict__ wb,
                        bf16 *__restrict__ wt, int update)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_total; t += (int64_t)gridDim.x * blockDim.x) {
        float p = w[t];
        if (update) {
            const float gt = g[t];
            const float mt = b1 * m[t] + (1.f - b1) * gt;
            const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
            m[t] = mt;
            v[t] = vt;
            const float mhat = mt / bc1, vhat = vt / bc2;
            p = p - lr * (mhat / (sqrtf(vhat) + eps) + wd * p);
            w[t] = p;
        }
        int k = 0;
        while (k < NT - 1 && t >= T.t[k + 1].off) ++k;
        const TensorDesc &d = T.t[k];
        if (d.wb_off >= 0) {
            const int64_t local = t - d.off;
            const int r = (int)(local / d.cols), c = (int)(local % d.cols);
            const bf16 b = __float2bfloat16_rn(p);
            wb[d.wb_off + local] = b;
            if (d.wt_off >= 0) wt[d.wt_off + (int64_t)c * d.rows + r] = b;
        }
    }
}

// per component sum and sum of squares (FP64) of samples[n][3*np3]
__global__ void k_moments(const float *__restrict__ samples, int64_t n, int np3, double *__restrict__ acc)
{
    __shared__ double s[6][256];
    double a[6] = {0, 0, 0, 0, 0, 0};
    const int64_t total = n * 3 * np3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)((t % (3 * np3)) / np3);
        const double x = samples[t];
        a[comp] += x;
        a[3 + comp] += x * x;
    }
    for (int q = 0; q < 6; ++q) s[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 6; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) atomicAdd(acc + q, s[q][0]);
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D map of a row-major BF16 matrix [rows][cols] (cols = K, contiguous), box 64 x box_rows
sem_status make_map(sem_ctx *ctx, CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int box_rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return sem_fail(ctx, SEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || cols % 64 != 0)
        return sem_fail(ctx, SEM_ERR_ARG, "GEMM operand not 16-byte aligned or K not a multiple of 64");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return sem_fail(ctx, SEM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SEM_OK;
}

unsigned grid_for(int64_t n, int threads, int sm)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 8LL * sm));
}

// sum of the `splits` partial arrays (stride floats apart) of a K-split product, in split order
// (deterministic), into out[0 .. n)
__global__ void k_split_reduce(const float *__restrict__ part, int splits, int64_t stride, int64_t n,
                               float *__restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float a = part[t];
        for (int z = 1; z < splits; ++z) a += part[z * stride + t];
        out[t] = a;
    }
}

// Plain arrival on an mbarrier (its expected count is the number of arriving warps).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Shared memory of the persistent GEMM: the TMA ring, then the epilogue warps' staging (the ring
// is busy with the next tile while a tile's epilogue runs, so the staging has its own room).
template <int BN, int NST>
struct PersistSmem {
    static constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr size_t RING = (size_t)NST * STAGE_BYTES;
    static constexpr size_t EPI = (size_t)4 * BN * 32 * 2 + (size_t)4 * 2 * 32 * EPI_RS * 2;
    static constexpr size_t BYTES = RING + EPI + 1024;
};

// The same product with one CTA per SM walking output tiles t = blockIdx.x, + gridDim.x, ...
// (tile t: M index t % mtiles, N index t / mtiles) and two TMEM accumulators of BN columns:
// while the epilogue warps drain accumulator i & 1 of tile i, the MMA warp fills the other one
// with tile i + 1, and the TMA ring runs on across tiles.  Barriers: full/empty for the ring,
// tfull[b] (MMA -> epilogue: accumulator b holds a finished tile) and tempty[b] (the four
// epilogue warps -> MMA: accumulator b has been read).  Every wait is bounded; on a time-out
// the kernel records SEM_ERR_TIMEOUT, every role stops, and before TMEM is freed the kernel waits
// (bounded) for its copies in flight and for every MMA it issued.  Results are those of
// k_gemm_bf16: each tile's products are accumulated in the same order.
template <int BN, int NST>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_bf16_p(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K,
                  int64_t mtiles, int64_t ntile, const __grid_constant__ EpiArgs P, int *err)
{
    using L = PersistSmem<BN, NST>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[NST], empty[NST], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ int s_consumed[NST];
    // SW128 tiles need 1024-byte alignment
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / BK;
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            s_consumed[s] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, 2 * BN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    int issued[NST] = {};
    if (warp == 0 && lane == 0) {
        // TMA producer: the ring's K slices of every tile this CTA walks
        int64_t g = 0;  // K slices issued so far
        for (int64_t t = blockIdx.x; t < ntile && !*(volatile int *)&s_abort; t += gridDim.x) {
            const int64_t mt = t % mtiles, nt = t / mtiles;
            for (int kb = 0; kb < nk; ++kb, ++g) {
                const int s = (int)(g % NST);
                const int64_t round = g / NST;
                if (round > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((round - 1) & 1), err)) {
                    s_abort = 1;
                    break;
                }
                if (*(volatile int *)&s_abort) break;
                uint8_t *a = smem + s * L::STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], L::STAGE_BYTES);
                tma_load_2d(a, &tmA, kb * BK, (int)(mt * BM), &full[s]);
                tma_load_2d(a + L::A_BYTES, &tmB, kb * BK, (int)(nt * BN), &full[s]);
                ++issued[s];
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tile i into accumulator i & 1, once the epilogue has read that accumulator's
        // previous tile
        constexpr uint32_t IDESC = tc::idesc_f16(BM, BN, true);
        int64_t g = 0;
        int i = 0;
        for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x, ++i) {
            const int b = i & 1, use = i >> 1;
            if (*(volatile int *)&s_abort ||
                (use > 0 && !mbar_wait_bounded(&tempty[b], (uint32_t)((use - 1) & 1), err))) {
                s_abort = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t tacc = tmem + (uint32_t)(b * BN);
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb, ++g) {
                const int s = (int)(g % NST);
                const int64_t round = g / NST;
                if (*(volatile int *)&s_abort || !mbar_wait_bounded(&full[s], (uint32_t)(round & 1), err)) {
                    s_abort = 1;
                    ok = false;
                    break;
                }
                s_consumed[s] = (int)(round + 1);
                tc::fence_after_sync();
                const uint32_t a = smem_u32(smem + s * L::STAGE_BYTES), bb = a + L::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc::mma_f16(tacc, tc::desc_k_sw128(a + kk * 32), tc::desc_k_sw128(bb + kk * 32), IDESC,
                                (kb | kk) != 0 ? 1u : 0u);
                tc::commit(&empty[s]);
            }
            if (!ok) break;
            tc::commit(&tfull[b]);
        }
        tc::commit(&done);  // arrives once every MMA this thread issued has completed
    } else if (warp >= 2) {
        // epilogue warps: warp q reads TMEM lane quarter q of each finished accumulator
        const int q = warp & 3;
        bf16 *tstage = reinterpret_cast<bf16 *>(smem + L::RING) + q * (BN * 32);
        bf16 *rs = reinterpret_cast<bf16 *>(smem + L::RING) + 4 * (BN * 32) + q * (2 * 32 * EPI_RS);
        int i = 0;
        for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x, ++i) {
            const int b = i & 1, use = i >> 1;
            // warp-uniform: the TMEM loads are collective over the warp
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[b], (uint32_t)(use & 1), err));
            if (!ok) s_abort = 1;
            if (!ok || __any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) break;
            tc::fence_after_sync();
            epilogue_tile<BN>(P, tmem + (uint32_t)(b * BN), t % mtiles, (int)(t / mtiles), 0, q, lane, tstage, rs);
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    // on an abort: wait (bounded) for this CTA's copies still in flight
    if (warp == 0 && lane == 0 && *(volatile int *)&s_abort) {
        for (int s = 0; s < NST; ++s)
            if (issued[s] > s_consumed[s]) mbar_wait_bounded(&full[s], s_consumed[s] & 1, nullptr);
    }
    // every MMA complete before TMEM is freed
    if (warp == 1 && lane == 0) mbar_wait_bounded(&done, 0, nullptr);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 2 * BN);
    }
}

struct GemmCfg {
    int bn, nst, split;
    int persist;  // 1: the persistent kernel (one CTA per SM walking the tiles), split 1 only
};

template <int BN, int NST>
sem_status launch_gemm(sem_ctx *ctx, const CUtensorMap &ta, const CUtensorMap &tb, int64_t M, int N, int K,
                       const EpiArgs &P, int split, const char *name)
{
    const size_t sm = (size_t)NST * (BM * BK * 2 + BN * BK * 2) + 1024;
    static KernelSetup ks;  // per instantiation and device
    SEM_TRY(kernel_setup(ctx, ks, k_gemm_bf16<BN, NST>, 0, sm));
    const dim3 grid((unsigned)(M / BM), (unsigned)(N / BN), (unsigned)split);
    SEM_TRACED(ctx, name, k_gemm_bf16<BN, NST><<<grid, GEMM_THREADS, sm, ctx->stream>>>(ta, tb, K, P, ctx->d_flag));
    return sem_cuda(ctx, cudaGetLastError(), "k_gemm_bf16 launch");
}

template <int BN, int NST>
sem_status launch_gemm_p(sem_ctx *ctx, const CUtensorMap &ta, const CUtensorMap &tb, int64_t M, int N, int K,
                         const EpiArgs &P, const char *name)
{
    constexpr size_t sm = PersistSmem<BN, NST>::BYTES;
    static KernelSetup ks;  // per instantiation and device
    SEM_TRY(kernel_setup(ctx, ks, k_gemm_bf16_p<BN, NST>, 0, sm));
    const int64_t mtiles = M / BM, ntile = mtiles * (N / BN);
    const unsigned grid = (unsigned)std::min<int64_t>(ntile, ctx->sm_count);
    SEM_TRACED(ctx, name, k_gemm_bf16_p<BN, NST><<<grid, GEMM_THREADS, sm, ctx->stream>>>(ta, tb, K, mtiles, ntile, P,
                                                                                         ctx->d_flag));
    return sem_cuda(ctx, cudaGetLastError(), "k_gemm_bf16_p launch");
}

// One product in configuration c: tensor maps for its tile shape, the K-split partials (weight
// gradients only) in the context's scratch and their ordered reduction.
sem_status run_gemm(sem_ctx *ctx, const void *A, const void *B, int64_t M, int N, int K, const EpiArgs &P,
                    GemmCfg c, const char *name)
{
    CUtensorMap ta, tb;
    SEM_TRY(make_map(ctx, &ta, A, M, K, BM));
    SEM_TRY(make_map(ctx, &tb, B, N, K, c.bn));
    EpiArgs Q = P;
    float *part = nullptr;
    const int64_t stride = M * (int64_t)P.ld_out;
    if (c.split > 1) {
        void *scr;
        SEM_TRY(sem_scratch_nogrow_in_capture(ctx, SCR_MISC, sizeof(float) * (size_t)(stride * c.split), &scr));
        part = static_cast<float *>(scr);
        Q.c32 = part;
        Q.split_stride = stride;
    }
    sem_status st;
#define SEM_GEMM_CASE(BNV, NSTV) \
    if (!c.persist && c.bn == BNV && c.nst == NSTV) st = launch_gemm<BNV, NSTV>(ctx, ta, tb, M, N, K, Q, c.split, name); else
#define SEM_GEMM_CASE_P(BNV, NSTV) \
    if (c.persist && c.split == 1 && c.bn == BNV && c.nst == NSTV) st = launch_gemm_p<BNV, NSTV>(ctx, ta, tb, M, N, K, Q, name); else
    SEM_GEMM_CASE(64, 3) SEM_GEMM_CASE(64, 4) SEM_GEMM_CASE(128, 3) SEM_GEMM_CASE(128, 4)
    SEM_GEMM_CASE(256, 3) SEM_GEMM_CASE(256, 4)
    SEM_GEMM_CASE_P(64, 3) SEM_GEMM_CASE_P(64, 4) SEM_GEMM_CASE_P(128, 3) SEM_GEMM_CASE_P(128, 4)
    return sem_fail(ctx, SEM_ERR_ARG, "no GEMM kernel for BN=%d, %d stages, persistent %d", c.bn, c.nst, c.persist);
#undef SEM_GEMM_CASE
#undef SEM_GEMM_CASE_P
    SEM_TRY(st);
    if (c.split > 1) {
        const int64_t n = P.m_valid * (int64_t)P.ld_out;
        SEM_TRACED(ctx, "k_split_reduce", k_split_reduce<<<grid_for(n, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
                                              part, c.split, stride, n, P.c32));
        SEM_CU(ctx, cudaGetLastError());
    }
    return SEM_OK;
}

// D = A B^T with A [M][K], B [N][K] (BF16, row-major), M % 128 == 0, N % 64 == 0, K % 64 == 0.
// The tile width, pipeline depth and (for FP32 weight gradients) K split come from the
// context's autotuner: the first product of a given (M, N, K, epilogue) runs every candidate on
// the call's own data (each twice, the second timed with CUDA events) and keeps the fastest;
// the candidates compute identical tiles, so the outputs do not depend on which one ran, except
// the order of the K-split partial sums.  Under stream capture, or with tuning off, the default
// (BN 128 when N allows, 4 stages, no split) is used.
sem_status gemm(sem_ctx *ctx, const void *A, const void *B, int64_t M, int N, int K, const EpiArgs &P,
                const char *name = "k_gemm_bf16")
{
    if (M % BM != 0 || K % BK != 0 || N % 64 != 0 || M <= 0 || N <= 0 || K <= 0)
        return sem_fail(ctx, SEM_ERR_ARG, "GEMM shape %lld x %d x %d not tileable", (long long)M, N, K);
    for (const auto &t : ctx->gemm_tune)
        if (t.M == M && t.N == N && t.K == K && t.mode == P.mode)
            return run_gemm(ctx, A, B, M, N, K, P, GemmCfg{t.bn, t.nst, t.split, t.persist}, name);
    const GemmCfg dflt{N % 128 == 0 ? 128 : 64, 4, 1, 0};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (!ctx->autotune || cs != cudaStreamCaptureStatusNone) return run_gemm(ctx, A, B, M, N, K, P, dflt, name);
    std::vector<GemmCfg> cand;
    const int nk = K / BK;
    const int64_t tiles = (M / BM) * (int64_t)(N / 128 > 0 ? N / 128 : 1);
    for (int bn : {64, 128, 256}) {
        if (N % bn != 0) continue;
        for (int nst : {3, 4}) {
            cand.push_back(GemmCfg{bn, nst, 1, 0});
            // the persistent form, whose epilogue overlaps the next tile's MMAs (its staging
            // beside the ring fits up to BN 128)
            if (bn <= 128) cand.push_back(GemmCfg{bn, nst, 1, 1});
            // K splits for the FP32 weight gradients, whose output tiles are few and K long
            // (K = the batch): at least 4 K blocks per split, at most 8 CTAs per SM in all
            if (P.mode == EPI_F32 && tiles < 2 * ctx->sm_count)
                for (int sp : {2, 4, 8, 16, 32})
                    if (nk / sp >= 4 && (M / BM) * (int64_t)(N / bn) * sp <= 8 * (int64_t)ctx->sm_count)
                        cand.push_back(GemmCfg{bn, nst, sp, 0});
        }
    }
    cudaEvent_t e0, e1;
    SEM_CU(ctx, cudaEventCreate(&e0));
    SEM_CU(ctx, cudaEventCreate(&e1));
    GemmCfg best = dflt;
    float best_ms = 1e30f;
    sem_status st = SEM_OK;
    for (const GemmCfg &c : cand) {
        for (int rep = 0; rep < 2 && st == SEM_OK; ++rep) {
            if (P.mode == EPI_LOSS) st = sem_cuda(ctx, cudaMemsetAsync(P.loss, 0, sizeof(float), ctx->stream), "memset");
            if (rep == 1 && st == SEM_OK) st = sem_cuda(ctx, cudaEventRecord(e0, ctx->stream), "event");
            if (st == SEM_OK) st = run_gemm(ctx, A, B, M, N, K, P, c, name);
            if (rep == 1 && st == SEM_OK) st = sem_cuda(ctx, cudaEventRecord(e1, ctx->stream), "event");
        }
        if (st != SEM_OK) break;
        float ms = 0.f;
        if ((st = sem_cuda(ctx, cudaEventSynchronize(e1), "event")) != SEM_OK) break;
        if ((st = sem_cuda(ctx, cudaEventElapsedTime(&ms, e0, e1), "event")) != SEM_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SEM_TRY(st);
    ctx->gemm_tune.push_back({M, N, K, P.mode, best.bn, best.nst, best.split, best.persist, best_ms});
    // the outputs (and the loss) of the chosen configuration
    if (P.mode == EPI_LOSS) SEM_CU(ctx, cudaMemsetAsync(P.loss, 0, sizeof(float), ctx->stream));
    return run_gemm(ctx, A, B, M, N, K, P, best, name);
}

EpiArgs epi(int mode, int64_t m_valid)
{
    EpiArgs e;
    memset(&e, 0, sizeof e);
    e.mode = mode;
    e.m_valid = m_valid;
    return e;
}


}  // namespace

// ==========================================================================================
// the autoencoder object
// ==========================================================================================
struct sem_ae {
    sem_ctx *ctx = nullptr;
    int Bp = 0;  // batch rows (multiple of 128)
    // flat FP32 arrays of the padded parameters: W1 [512][1536], b1 [512], W2 [64][512],
    // b2 [64], W3 [512][64], b3 [512], W4 [1536][512], b4 [1536]
    AdamTable tab;
    int64_t n_param = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;
    int64_t n_wb = 0;
    float mean[3] = {0, 0, 0}, stdv[3] = {1, 1, 1};
    int64_t step = 0;
    float *loss = nullptr;  // device
    // activations (BF16): rows Bp
    bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *A1 = nullptr, *A1T = nullptr, *Z = nullptr, *ZT = nullptr;
    bf16 *H3 = nullptr, *A3 = nullptr, *A3T = nullptr, *dY = nullptr, *dYT = nullptr, *dH3 = nullptr, *dH3T = nullptr;
    bf16 *dZ = nullptr, *dZT = nullptr, *dH1 = nullptr, *dH1T = nullptr;
    void *arena = nullptr;
    int64_t bytes = 0;
};

namespace {
constexpr int D_IN = 1536, D_H = 512, D_ZP = 64, NP3_AE = 512;  // widths (latent 48 padded to 64)
// unpadded parameter shapes, in the order of the flat host arrays
const int kShape[8][2] = {{512, 1536}, {512, 1}, {48, 512}, {48, 1}, {512, 48}, {512, 1}, {1536, 512}, {1536, 1}};
// padded shapes on the device
const int kPad[8][2] = {{512, 1536}, {512, 1}, {64, 512}, {64, 1}, {512, 64}, {512, 1}, {1536, 512}, {1536, 1}};

int64_t host_param_count()
{
    int64_t n = 0;
    for (auto &s : kShape) n += (int64_t)s[0] * s[1];
    return n;
}

sem_status ae_forward(sem_ae *ae, int B, bool want_loss, bool training)
{
    sem_ctx *ctx = ae->ctx;
    const int Bp = ae->Bp;
    const TensorDesc *T = ae->tab.t;
    const bf16 *W1 = ae->wb + T[0].wb_off, *W2 = ae->wb + T[2].wb_off, *W3 = ae->wb + T[4].wb_off,
               *W4 = ae->wb + T[6].wb_off;
    EpiArgs e = epi(EPI_BIAS_GELU, Bp);
    e.bias = ae->w + T[1].off;
    e.out = ae->H1;
    e.aux = ae->A1;
    e.ld_out = D_H;
    e.out_t = ae->A1T;
    e.ld_t = Bp;
    SEM_TRY(gemm(ctx, ae->X, W1, Bp, D_H, D_IN, e, "k_gemm_bf16 fwd1"));
    e = epi(EPI_BIAS, Bp);
    e.bias = ae->w + T[3].off;
    e.out = ae->Z;
    e.ld_out = D_ZP;
    e.out_t = ae->ZT;
    e.ld_t = Bp;
    SEM_TRY(gemm(ctx, ae->A1, W2, Bp, D_ZP, D_H, e, "k_gemm_bf16 fwd2"));
    e = epi(EPI_BIAS_GELU, Bp);
    e.bias = ae->w + T[5].off;
    e.out = ae->H3;
    e.aux = ae->A3;
    e.ld_out = D_H;
    e.out_t = ae->A3T;
    e.ld_t = Bp;
    SEM_TRY(gemm(ctx, ae->Z, W3, Bp, D_H, D_ZP, e, "k_gemm_bf16 fwd3"));
    if (!want_loss) return SEM_OK;
    e = epi(EPI_LOSS, B);
    e.bias = ae->w + T[7].off;
    e.out = ae->dY;
    e.ld_out = D_IN;
    e.out_t = ae->dYT;
    e.ld_t = Bp;
    e.in = ae->X;
    e.ld_in = D_IN;
    e.loss = ae->loss;
    e.scale = 2.0f / ((float)B * (float)D_IN);
    SEM_CU(ctx, cudaMemsetAsync(ae->loss, 0, sizeof(float), ctx->stream));
    SEM_TRY(gemm(ctx, ae->A3, W4, Bp, D_IN, D_H, e, "k_gemm_bf16 fwd4"));
    (void)training;
    return SEM_OK;
}

sem_status ae_backward(sem_ae *ae, int B)
{
    sem_ctx *ctx = ae->ctx;
    const int Bp = ae->Bp;
    const TensorDesc *T = ae->tab.t;
    const bf16 *W2t = ae->wt + T[2].wt_off, *W3t = ae->wt + T[4].wt_off, *W4t = ae->wt + T[6].wt_off;
    float *g = ae->g;
    // layer 4: dA3 = dY W4 -> dH3 = dA3 gelu'(H3); dW4 = dY^T A3
    EpiArgs e = epi(EPI_DGELU, Bp);
    e.out = ae->dH3;
    e.ld_out = D_H;
    e.out_t = ae->dH3T;
    e.ld_t = Bp;
    e.in = ae->H3;
    e.ld_in = D_H;
    SEM_TRY(gemm(ctx, ae->dY, W4t, Bp, D_H, D_IN, e, "k_gemm_bf16 dx4"));
    e = epi(EPI_F32, D_IN);
    e.c32 = g + T[6].off;
    e.ld_out = D_H;
    SEM_TRY(gemm(ctx, ae->dYT, ae->A3T, D_IN, D_H, Bp, e, "k_gemm_bf16 dw4"));
    // layer 3: dZ = dH3 W3; dW3 = dH3^T Z
    e = epi(EPI_PLAIN, Bp);
    e.out = ae->dZ;
    e.ld_out = D_ZP;
    e.out_t = ae->dZT;
    e.ld_t = Bp;
    SEM_TRY(gemm(ctx, ae->dH3, W3t, Bp, D_ZP, D_H, e, "k_gemm_bf16 dx3"));
    e = epi(EPI_F32, D_H);
    e.c32 = g + T[4].off;
    e.ld_out = D_ZP;
    SEM_TRY(gemm(ctx, ae->dH3T, ae->ZT, D_H, D_ZP, Bp, e, "k_gemm_bf16 dw3"));
    // layer 2: dA1 = dZ W2 -> dH1 = dA1 gelu'(H1); dW2 = dZ^T A1 (dZ^T padded to 128 rows)
    e = epi(EPI_DGELU, Bp);
    e.out = ae->dH1;
    e.ld_out = D_H;
    e.out_t = ae->dH1T;
    e.ld_t = Bp;
    e.in = ae->H1;
    e.ld_in = D_H;
    SEM_TRY(gemm(ctx, ae->dZ, W2t, Bp, D_H, D_ZP, e, "k_gemm_bf16 dx2"));
    e = epi(EPI_F32, D_ZP);
    e.c32 = g + T[2].off;
    e.ld_out = D_H;
    SEM_TRY(gemm(ctx, ae->dZT, ae->A1T, 128, D_H, Bp, e, "k_gemm_bf16 dw2"));
    // layer 1: dW1 = dH1^T X
    e = epi(EPI_F32, D_H);
    e.c32 = g + T[0].off;
    e.ld_out = D_IN;
    SEM_TRY(gemm(ctx, ae->dH1T, ae->XT, D_H, D_IN, Bp, e, "k_gemm_bf16 dw1"));
    // bias gradients: row sums of the transposed gradients (the padding columns are zero)
    SEM_TRACED(ctx, "k_rowsum", k_rowsum<<<(D_IN + 7) / 8, 256, 0, ctx->stream>>>(ae->dYT, D_IN, B, Bp, g + T[7].off));
    SEM_TRACED(ctx, "k_rowsum", k_rowsum<<<(D_H + 7) / 8, 256, 0, ctx->stream>>>(ae->dH3T, D_H, B, Bp, g + T[5].off));
    SEM_TRACED(ctx, "k_rowsum", k_rowsum<<<(D_ZP + 7) / 8, 256, 0, ctx->stream>>>(ae->dZT, D_ZP, B, Bp, g + T[3].off));
    SEM_TRACED(ctx, "k_rowsum", k_rowsum<<<(D_H + 7) / 8, 256, 0, ctx->stream>>>(ae->dH1T, D_H, B, Bp, g + T[1].off));
    return sem_cuda(ctx, cudaGetLastError(), "k_rowsum launch");
}

sem_status ae_refresh_copies(sem_ae *ae, bool update, float lr, float b1, float b2, float eps, float wd)
{
    sem_ctx *ctx = ae->ctx;
    float bc1 = 1.f, bc2 = 1.f;
    if (update) {
        ae->step += 1;
        bc1 = (float)(1.0 - pow((double)b1, (double)ae->step));
        bc2 = (float)(1.0 - pow((double)b2, (double)ae->step));
    }
    SEM_TRACED(ctx, "k_adamw", k_adamw<<<grid_for(ae->n_param, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
                                   ae->tab, ae->n_param, ae->w, ae->m, ae->v, ae->g, lr, b1, b2, eps, wd, bc1, bc2,
                                   ae->wb, ae->wt, update ? 1 : 0));
    return sem_cuda(ctx, cudaGetLastError(), "k_adamw launch");
}

sem_status ae_pack_samples(sem_ae *ae, const float *samples, int64_t n_samples, const int64_t *idx, int B)
{
    sem_ctx *ctx = ae->ctx;
    const dim3 pg(D_IN / 32, ae->Bp / 32);
    SEM_TRACED(ctx, "k_pack", k_pack<<<pg, 256, 0, ctx->stream>>>(
                                  samples, idx, n_samples, nullptr, nullptr, nullptr, 0, B, ae->Bp, NP3_AE, ae->mean[0],
                                  ae->mean[1], ae->mean[2], 1.f / ae->stdv[0], 1.f / ae->stdv[1], 1.f / ae->stdv[2],
                                  ae->X, ae->XT, ctx->d_flag));
    return sem_cuda(ctx, cudaGetLastError(), "k_pack launch");
}

sem_status check_ae(sem_ae *ae, const char *fn)
{
    if (!ae) return SEM_ERR_ARG;
    SEM_CU(ae->ctx, cudaSetDevice(ae->ctx->device));
    (void)fn;
    return SEM_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
sem_status sem_ae_create(sem_ctx *ctx, int batch, sem_ae **out)
{
    if (!ctx || !out) return SEM_ERR_ARG;
    *out = nullptr;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (batch < 128 || batch % 128 != 0 || batch > (1 << 20))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_create: batch %d is not a positive multiple of 128", batch);
    sem_ae *ae = new sem_ae();
    ae->ctx = ctx;
    ae->Bp = batch;
    // parameter table (padded shapes)
    int64_t off = 0, wboff = 0;
    for (int k = 0; k < NT; ++k) {
        TensorDesc &d = ae->tab.t[k];
        d.off = off;
        d.rows = kPad[k][0];
        d.cols = kPad[k][1];
        off += (int64_t)d.rows * d.cols;
        if (kPad[k][1] > 1) {
            d.wb_off = wboff;
            wboff += (int64_t)d.rows * d.cols;
        } else {
            d.wb_off = -1;
        }
    }
    ae->n_param = off;
    ae->n_wb = wboff;
    for (int k = 0; k < NT; ++k) ae->tab.t[k].wt_off = ae->tab.t[k].wb_off;  // same offsets in the transpose array
    // one arena: params, moments, gradients, BF16 copies, activations
    const int Bp = batch;
    const size_t fbytes = sizeof(float) * (size_t)ae->n_param;
    const size_t wbytes = sizeof(bf16) * (size_t)ae->n_wb;
    struct Piece {
        void **dst;
        size_t bytes;
    };
    const size_t r = sizeof(bf16) * (size_t)Bp;
    std::vector<Piece> pieces = {
        {(void **)&ae->w, fbytes}, {(void **)&ae->m, fbytes}, {(void **)&ae->v, fbytes}, {(void **)&ae->g, fbytes},
        {(void **)&ae->wb, wbytes}, {(void **)&ae->wt, wbytes}, {(void **)&ae->loss, 256},
        {(void **)&ae->X, r * D_IN}, {(void **)&ae->XT, r * D_IN}, {(void **)&ae->H1, r * D_H},
        {(void **)&ae->A1, r * D_H}, {(void **)&ae->A1T, r * D_H}, {(void **)&ae->Z, r * D_ZP},
        {(void **)&ae->ZT, r * D_ZP}, {(void **)&ae->H3, r * D_H}, {(void **)&ae->A3, r * D_H},
        {(void **)&ae->A3T, r * D_H}, {(void **)&ae->dY, r * D_IN}, {(void **)&ae->dYT, r * D_IN},
        {(void **)&ae->dH3, r * D_H}, {(void **)&ae->dH3T, r * D_H}, {(void **)&ae->dZ, r * D_ZP},
        {(void **)&ae->dZT, r * 128}, {(void **)&ae->dH1, r * D_H}, {(void **)&ae->dH1T, r * D_H}};
    size_t total = 0;
    for (auto &p : pieces) total += (p.bytes + 1023) / 1024 * 1024;
    cudaError_t e = cudaMalloc(&ae->arena, total);
    if (e != cudaSuccess) {
        delete ae;
        return sem_cuda(ctx, e, "sem_ae_create: cudaMalloc");
    }
    ctx->mem_add((int64_t)total);
    ae->bytes = (int64_t)total;
    size_t at = 0;
    for (auto &p : pieces) {
        *p.dst = static_cast<char *>(ae->arena) + at;
        at += (p.bytes + 1023) / 1024 * 1024;
    }
    // everything starts at zero (padding rows/columns of weights and dZ^T stay zero)
    e = cudaMemsetAsync(ae->arena, 0, total, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(ae->arena);
        ctx->mem_add(-(int64_t)total);
        delete ae;
        return sem_cuda(ctx, e, "sem_ae_create: memset");
    }
    *out = ae;
    return SEM_OK;
}

void sem_ae_destroy(sem_ae *ae)
{
    if (!ae) return;
    cudaSetDevice(ae->ctx->device);
    cudaStreamSynchronize(ae->ctx->stream);
    if (ae->arena) cudaFree(ae->arena);
    ae->ctx->mem_add(-ae->bytes);
    delete ae;
}

int64_t sem_ae_param_count(void) { return host_param_count(); }

// host flat unpadded <-> device padded
static void scatter_params(const float *host, std::vector<float> &dev, const AdamTable &tab)
{
    int64_t h = 0;
    for (int k = 0; k < NT; ++k) {
        const TensorDesc &d = tab.t[k];
        for (int rr = 0; rr < kShape[k][0]; ++rr)
            for (int cc = 0; cc < kShape[k][1]; ++cc) dev[d.off + (int64_t)rr * d.cols + cc] = host[h++];
    }
}

static void gather_params(const std::vector<float> &dev, float *host, const AdamTable &tab)
{
    int64_t h = 0;
    for (int k = 0; k < NT; ++k) {
        const TensorDesc &d = tab.t[k];
        for (int rr = 0; rr < kShape[k][0]; ++rr)
            for (int cc = 0; cc < kShape[k][1]; ++cc) host[h++] = dev[d.off + (int64_t)rr * d.cols + cc];
    }
}

static sem_status copy_flat(sem_ae *ae, float *dev_arr, const float *host, int64_t n, bool to_dev, float *host_out)
{
    sem_ctx *ctx = ae->ctx;
    if (n != host_param_count())
        return sem_fail(ctx, SEM_ERR_ARG, "autoencoder arrays hold %lld values, got %lld", (long long)host_param_count(),
                        (long long)n);
    std::vector<float> buf((size_t)ae->n_param, 0.f);
    if (to_dev) {
        scatter_params(host, buf, ae->tab);
        SEM_CU(ctx, cudaMemcpyAsync(dev_arr, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice, ctx->stream));
        SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    } else {
        SEM_CU(ctx, cudaMemcpyAsync(buf.data(), dev_arr, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost, ctx->stream));
        SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
        gather_params(buf, host_out, ae->tab);
    }
    return SEM_OK;
}

sem_status sem_ae_set_params(sem_ae *ae, const float *host, int64_t n)
{
    SEM_TRY(check_ae(ae, "sem_ae_set_params"));
    if (!host) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_set_params: host is NULL");
    SEM_TRY(copy_flat(ae, ae->w, host, n, true, nullptr));
    return ae_refresh_copies(ae, false, 0.f, 0.f, 0.f, 0.f, 0.f);
}

sem_status sem_ae_get_params(sem_ae *ae, float *host, int64_t n)
{
    SEM_TRY(check_ae(ae, "sem_ae_get_params"));
    if (!host) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_get_params: host is NULL");
    return copy_flat(ae, ae->w, nullptr, n, false, host);
}

sem_status sem_ae_get_state(sem_ae *ae, float *m_host, float *v_host, int64_t n, int64_t *step)
{
    SEM_TRY(check_ae(ae, "sem_ae_get_state"));
    if (!m_host || !v_host || !step) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_get_state: NULL argument");
    SEM_TRY(copy_flat(ae, ae->m, nullptr, n, false, m_host));
    SEM_TRY(copy_flat(ae, ae->v, nullptr, n, false, v_host));
    *step = ae->step;
    return SEM_OK;
}

sem_status sem_ae_set_state(sem_ae *ae, const float *m_host, const float *v_host, int64_t n, int64_t step)
{
    SEM_TRY(check_ae(ae, "sem_ae_set_state"));
    if (!m_host || !v_host || step < 0) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_set_state: bad argument");
    SEM_TRY(copy_flat(ae, ae->m, m_host, n, true, nullptr));
    SEM_TRY(copy_flat(ae, ae->v, v_host, n, true, nullptr));
    ae->step = step;
    return SEM_OK;
}

sem_status sem_ae_set_normalization(sem_ae *ae, const float mean[3], const float stdv[3])
{
    SEM_TRY(check_ae(ae, "sem_ae_set_normalization"));
    if (!mean || !stdv) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_set_normalization: NULL");
    for (int c = 0; c < 3; ++c) {
        if (!(stdv[c] > 0.f) || !isfinite(mean[c]))
            return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_set_normalization: std must be positive");
        ae->mean[c] = mean[c];
        ae->stdv[c] = stdv[c];
    }
    return SEM_OK;
}

sem_status sem_ae_get_normalization(sem_ae *ae, float mean[3], float stdv[3])
{
    SEM_TRY(check_ae(ae, "sem_ae_get_normalization"));
    if (!mean || !stdv) return sem_fail(ae->ctx, SEM_ERR_ARG, "sem_ae_get_normalization: NULL");
    for (int c = 0; c < 3; ++c) {
        mean[c] = ae->mean[c];
        stdv[c] = ae->stdv[c];
    }
    return SEM_OK;
}

sem_status sem_ae_fit_normalization(sem_ae *ae, const float *samples, int64_t n)
{
    SEM_TRY(check_ae(ae, "sem_ae_fit_normalization"));
    sem_ctx *ctx = ae->ctx;
    if (!samples || n < 2) return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_fit_normalization: need >= 2 samples");
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_MISC, 6 * sizeof(double), &scr));
    double *acc = static_cast<double *>(scr);
    SEM_CU(ctx, cudaMemsetAsync(acc, 0, 6 * sizeof(double), ctx->stream));
    SEM_TRACED(ctx, "k_moments", k_moments<<<grid_for(n * 3 * NP3_AE, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
                                     samples, n, NP3_AE, acc));
    SEM_CU(ctx, cudaGetLastError());
    double h[6];
    SEM_CU(ctx, cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    // per-component means; one common scale, the root of the mean per-component variance, so a
    // component that carries only noise (w of a Taylor-Green field) is not blown up to unit
    // variance
    const double cnt = (double)n * NP3_AE;
    double var = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double mu = h[c] / cnt;
        var += (h[3 + c] / cnt - mu * mu) / 3.0;
        ae->mean[c] = (float)mu;
    }
    const float sd = (float)sqrt(var > 1e-30 ? var : 1e-30);
    for (int c = 0; c < 3; ++c) ae->stdv[c] = sd;
    return SEM_OK;
}

sem_status sem_ae_loss_grad(sem_ae *ae, const float *samples, int64_t n_samples, const int64_t *idx, int B,
                            float *loss_host, float *grad_host, int64_t n)
{
    SEM_TRY(check_ae(ae, "sem_ae_loss_grad"));
    sem_ctx *ctx = ae->ctx;
    if (!samples || !idx || B < 1 || B > ae->Bp || n_samples < 1)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_loss_grad: need samples, idx and 1 <= B <= %d", ae->Bp);
    SEM_TRY(ae_pack_samples(ae, samples, n_samples, idx, B));
    SEM_TRY(ae_forward(ae, B, true, true));
    SEM_TRY(ae_backward(ae, B));
    if (loss_host) {
        float l = 0.f;
        SEM_CU(ctx, cudaMemcpyAsync(&l, ae->loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
        *loss_host = l / ((float)B * (float)D_IN);
    }
    if (grad_host) SEM_TRY(copy_flat(ae, ae->g, nullptr, n, false, grad_host));
    return SEM_OK;
}

sem_status sem_ae_train_step(sem_ae *ae, const float *samples, int64_t n_samples, const int64_t *idx, int B,
                             float lr, float beta1, float beta2, float eps, float weight_decay, float *loss_dev)
{
    SEM_TRY(check_ae(ae, "sem_ae_train_step"));
    sem_ctx *ctx = ae->ctx;
    if (!samples || !idx || B < 1 || B > ae->Bp || n_samples < 1)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_train_step: need samples, idx and 1 <= B <= %d", ae->Bp);
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_train_step: bad hyper-parameters");
    SEM_TRY(ae_pack_samples(ae, samples, n_samples, idx, B));
    SEM_TRY(ae_forward(ae, B, true, true));
    SEM_TRY(ae_backward(ae, B));
    if (loss_dev)
        SEM_CU(ctx, cudaMemcpyAsync(loss_dev, ae->loss, sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    return ae_refresh_copies(ae, true, lr, beta1, beta2, eps, weight_decay);
}

sem_status sem_ae_encode(sem_ae *ae, const float *u, const float *v, const float *w, int64_t E, uint16_t *latent)
{
    SEM_TRY(check_ae(ae, "sem_ae_encode"));
    sem_ctx *ctx = ae->ctx;
    if (E < 0 || (E > 0 && (!u || !v || !w || !latent))) return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_encode: bad arguments");
    if ((reinterpret_cast<uintptr_t>(latent) & 15u) != 0)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_encode: latent must be 16-byte aligned");
    const int Bp = ae->Bp;
    for (int64_t e0 = 0; e0 < E; e0 += Bp) {
        const int B = (int)std::min<int64_t>(Bp, E - e0);
        const dim3 pg(D_IN / 32, Bp / 32);
        SEM_TRACED(ctx, "k_pack", k_pack<<<pg, 256, 0, ctx->stream>>>(
                                      nullptr, nullptr, 0, u, v, w, e0, B, Bp, NP3_AE, ae->mean[0], ae->mean[1],
                                      ae->mean[2], 1.f / ae->stdv[0], 1.f / ae->stdv[1], 1.f / ae->stdv[2], ae->X,
                                      nullptr, nullptr));
        SEM_CU(ctx, cudaGetLastError());
        const TensorDesc *T = ae->tab.t;
        EpiArgs e = epi(EPI_BIAS_GELU, Bp);
        e.bias = ae->w + T[1].off;
        e.out = ae->H1;
        e.aux = ae->A1;
        e.ld_out = D_H;
        e.out_t = ae->A1T;
        e.ld_t = Bp;
        SEM_TRY(gemm(ctx, ae->X, ae->wb + T[0].wb_off, Bp, D_H, D_IN, e));
        e = epi(EPI_LATENT, B);
        e.bias = ae->w + T[3].off;
        e.out = reinterpret_cast<bf16 *>(latent) + e0 * 48;
        SEM_TRY(gemm(ctx, ae->A1, ae->wb + T[2].wb_off, Bp, D_ZP, D_H, e));
    }
    return SEM_OK;
}

sem_status sem_ae_decode(sem_ae *ae, const uint16_t *latent, int64_t E, float *u, float *v, float *w)
{
    SEM_TRY(check_ae(ae, "sem_ae_decode"));
    sem_ctx *ctx = ae->ctx;
    if (E < 0 || (E > 0 && (!u || !v || !w || !latent))) return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_decode: bad arguments");
    for (const float *p : {u, v, w})
        if (E > 0 && (reinterpret_cast<uintptr_t>(p) & 15u) != 0)
            return sem_fail(ctx, SEM_ERR_ARG, "sem_ae_decode: fields must be 16-byte aligned");
    const int Bp = ae->Bp;
    const TensorDesc *T = ae->tab.t;
    for (int64_t e0 = 0; e0 < E; e0 += Bp) {
        const int B = (int)std::min<int64_t>(Bp, E - e0);
        SEM_TRACED(ctx, "k_latent_in", k_latent_in<<<grid_for((int64_t)Bp * 64, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
                                           reinterpret_cast<const bf16 *>(latent), e0, B, Bp, ae->Z));
        SEM_CU(ctx, cudaGetLastError());
        EpiArgs e = epi(EPI_BIAS_GELU, Bp);
        e.bias = ae->w + T[5].off;
        e.out = ae->H3;
        e.aux = ae->A3;
        e.ld_out = D_H;
        e.out_t = ae->A3T;
        e.ld_t = Bp;
        SEM_TRY(gemm(ctx, ae->Z, ae->wb + T[4].wb_off, Bp, D_H, D_ZP, e));
        e = epi(EPI_DECODE, B);
        e.bias = ae->w + T[7].off;
        e.fields[0] = u + e0 * NP3_AE;
        e.fields[1] = v + e0 * NP3_AE;
        e.fields[2] = w + e0 * NP3_AE;
        e.np3 = NP3_AE;
        for (int c = 0; c < 3; ++c) {
            e.mean[c] = ae->mean[c];
            e.stdv[c] = ae->stdv[c];
        }
        SEM_TRY(gemm(ctx, ae->A3, ae->wb + T[6].wb_off, Bp, D_IN, D_H, e));
    }
    return SEM_OK;
}

sem_status sem_gemm_bf16(sem_ctx *ctx, const uint16_t *A, const uint16_t *B, int64_t M, int N, int K, float *C)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (!A || !B || !C) return sem_fail(ctx, SEM_ERR_ARG, "sem_gemm_bf16: NULL operand");
    if ((reinterpret_cast<uintptr_t>(C) & 15u) != 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_gemm_bf16: C not 16-byte aligned");
    EpiArgs e = epi(EPI_F32, M);
    e.c32 = C;
    e.ld_out = N;
    return gemm(ctx, A, B, M, N, K, e);
}

sem_status sem_autotune_set(sem_ctx *ctx, int on)
{
    if (!ctx) return SEM_ERR_ARG;
    ctx->autotune = on != 0;
    if (!on) {
        ctx->gemm_tune.clear();
        ctx->emit_tune.clear();
        ctx->width_tune.clear();
    }
    return SEM_OK;
}

sem_status sem_autotune_emit_entry(sem_ctx *ctx, int k, int *N, int64_t *E, int *niso, int *units, float *ms)
{
    if (!ctx || !N || !E || !niso || !units || !ms) return SEM_ERR_ARG;
    if (k < 0 || k >= (int)ctx->emit_tune.size())
        return sem_fail(ctx, SEM_ERR_ARG, "sem_autotune_emit_entry: index %d outside [0, %d)", k,
                        (int)ctx->emit_tune.size());
    const auto &t = ctx->emit_tune[k];
    *N = t.N;
    *E = t.E;
    *niso = t.niso;
    *units = t.units;
    *ms = t.ms;
    return SEM_OK;
}

sem_status sem_autotune_width_entry(sem_ctx *ctx, int k, int *kind, int *N, int64_t *size, int *width, float *ms)
{
    if (!ctx || !kind || !N || !size || !width || !ms) return SEM_ERR_ARG;
    if (k < 0 || k >= (int)ctx->width_tune.size())
        return sem_fail(ctx, SEM_ERR_ARG, "sem_autotune_width_entry: index %d outside [0, %d)", k,
                        (int)ctx->width_tune.size());
    const auto &t = ctx->width_tune[k];
    *kind = t.kind;
    *N = t.N;
    *size = t.size;
    *width = t.width;
    *ms = t.ms;
    return SEM_OK;
}

sem_status sem_autotune_entry(sem_ctx *ctx, int k, int64_t *M, int *N, int *K, int *mode, int *bn, int *stages,
                              int *split, int *persistent, float *ms)
{
    if (!ctx || !M || !N || !K || !mode || !bn || !stages || !split || !ms) return SEM_ERR_ARG;
    if (k < 0 || k >= (int)ctx->gemm_tune.size())
        return sem_fail(ctx, SEM_ERR_ARG, "sem_autotune_entry: index %d outside [0, %d)", k, (int)ctx->gemm_tune.size());
    const auto &t = ctx->gemm_tune[k];
    *M = t.M;
    *N = t.N;
    *K = t.K;
    *mode = t.mode;
    *bn = t.bn;
    *stages = t.nst;
    *split = t.split;
    if (persistent) *persistent = t.persist;
    *ms = t.ms;
    return SEM_OK;
}
