// bbe_surrogate.cu -- the win-probability surrogate network (include/bbe_surrogate.h):
// forward, backward and Adam kernels and the C ABI around them.
//
// Work is cut into tiles of at most 128 competitor rows holding whole races (at most 64),
// so that the mean-pooled context and the per-race softmax stay inside one thread block.
// A block of 8 warps processes one tile; warp w owns rows 16w..16w+15.  Every matrix
// product runs on the tensor cores with mma.sync m16n8k16 (bfloat16 operands staged in
// shared memory, loaded with ldmatrix, float32 accumulators in registers):
//   forward   Y[rows][out] = X[rows][in] . W[out][in]^T
//   backward  dX = dY . W,   dW += dY^T . X  (reduced over the tile's rows, then added to
//             the float32 gradient with vector atomics)
// The layer weights are streamed into shared memory one layer at a time.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "bbe_internal.h"
#include "bbe_surrogate.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int H = 128;        // hidden width
constexpr int KIN = 16;       // input features padded to one k-step
constexpr int FIN = 14;       // input features in use (raw and derived)
constexpr int RAW = 5;        // raw per-competitor quantities (range-checked at inference)
constexpr int TILE = 128;     // rows per tile
constexpr int MAX_STATES = 64;
constexpr int NTHREADS = 256;
constexpr float L_SCALE = 5000.0f;

// flat parameter layout (floats)
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * KIN;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H * H;
constexpr int OFF_W4 = OFF_B3 + H;
constexpr int OFF_B4 = OFF_W4 + H * 2 * H;
constexpr int OFF_W5 = OFF_B4 + H;
constexpr int OFF_B5 = OFF_W5 + H;
constexpr int N_PARAMS = OFF_B5 + 1;

// shared-memory row strides (bf16 elements): +8 keeps ldmatrix rows on distinct banks
constexpr int LD_IN = KIN + 8;   // 24
constexpr int LD_H = H + 8;      // 136
constexpr int LD_2H = 2 * H + 8; // 264

// per-tile training workspace (global memory)
constexpr size_t WS_X = size_t(TILE) * KIN;   // bf16
constexpr size_t WS_H = size_t(TILE) * H;     // bf16, one per h1, h2, h3, u

struct SgTile {
    int32_t s0;     // first position in the order array
    int32_t ns;     // races in the tile
    int32_t nrows;  // competitor rows
    int32_t pad;
};

struct SgArgs {
    const bf16 *wb;        // bfloat16 copy of the parameters (flat layout)
    const float *wf;       // float32 master parameters (biases and w5 are read from here)
    const SgTile *tiles;
    const int32_t *order;  // race indices in tile order
    bbe::DevBatch b;
    float *probs;          // forward output per competitor (batch order) or null
    const float *target;   // training targets per competitor (batch order)
    float inv_races;       // 1 / races in the step
    float *loss_acc;       // training: mean loss accumulator (device scalar) or null
    float *grad;           // training: float32 gradient (flat layout)
    bf16 *ws;              // training workspace, tile-major
    float *ws_dlogit;      // training: d loss / d logit per tile row
    int train;
};

// ------------------------------------------------------------------ tensor-core helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int NT>
__device__ __forceinline__ void zero_acc(float (&acc)[NT][4])
{
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
}

// acc[16 rows][8*NT] += A[16 rows][K] . W[8*NT][K]^T   (A: this warp's rows; W: [out][in])
template <int NT, int K>
__device__ __forceinline__ void gemm_xwT(float (&acc)[NT][4], const bf16 *A, int lda, const bf16 *W, int ldw,
                                         int lane)
{
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        ldsm_x4(a, A + (lane & 15) * lda + k0 + (lane >> 4) * 8);
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            const int mi = lane >> 3;
            uint32_t bq[4];
            ldsm_x4(bq, W + (j * 8 + (lane & 7) + (mi >> 1) * 8) * ldw + k0 + (mi & 1) * 8);
            mma16816(acc[j], a, bq[0], bq[1]);
            mma16816(acc[j + 1], a, bq[2], bq[3]);
        }
    }
}

// acc[16 rows][8*NT] += dY[16 rows][N] . W[N][8*NT]   (W: [reduction][out] block of [out..][in])
template <int NT, int N>
__device__ __forceinline__ void gemm_dyW(float (&acc)[NT][4], const bf16 *dY, int ldy, const bf16 *W, int ldw,
                                         int lane)
{
#pragma unroll 2
    for (int n0 = 0; n0 < N; n0 += 16) {
        uint32_t a[4];
        ldsm_x4(a, dY + (lane & 15) * ldy + n0 + (lane >> 4) * 8);
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            const int mi = lane >> 3;
            uint32_t bq[4];
            ldsm_x4_t(bq, W + (n0 + (lane & 7) + (mi & 1) * 8) * ldw + j * 8 + (mi >> 1) * 8);
            mma16816(acc[j], a, bq[0], bq[1]);
            mma16816(acc[j + 1], a, bq[2], bq[3]);
        }
    }
}

// acc[16 outs (n0..n0+15)][8*NT] += sum over the tile's 128 rows of dY[row][n] X[row][k]
template <int NT>
__device__ __forceinline__ void gemm_dyT_x(float (&acc)[NT][4], const bf16 *dY, int ldy, int n0, const bf16 *X,
                                           int ldx, int lane)
{
    const int mi = lane >> 3;
#pragma unroll 2
    for (int m0 = 0; m0 < TILE; m0 += 16) {
        uint32_t a[4];
        ldsm_x4_t(a, dY + (m0 + (lane & 7) + (mi >> 1) * 8) * ldy + n0 + (mi & 1) * 8);
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            uint32_t bq[4];
            ldsm_x4_t(bq, X + (m0 + (lane & 7) + (mi & 1) * 8) * ldx + j * 8 + (mi >> 1) * 8);
            mma16816(acc[j], a, bq[0], bq[1]);
            mma16816(acc[j + 1], a, bq[2], bq[3]);
        }
    }
}

// copy a [128][K] bf16 matrix (row stride K in global) into shared memory with stride ld
template <int K>
__device__ __forceinline__ void load_rows(bf16 *dst, int ld, const bf16 *src, int tid)
{
    constexpr int VPR = K / 8;  // 16-byte vectors per row
    for (int i = tid; i < TILE * VPR; i += NTHREADS) {
        const int r = i / VPR, v = i - r * VPR;
        *reinterpret_cast<uint4 *>(dst + r * ld + v * 8) = *reinterpret_cast<const uint4 *>(src + size_t(r) * K + v * 8);
    }
}

// gradient of a [128 outs][K] block: accumulator rows n0 + g (+8), columns j*8 + 2t (+1)
template <int NT>
__device__ __forceinline__ void atomic_add_block(float *g, int ldg, int n0, int col0, const float (&acc)[NT][4],
                                                 int lane)
{
    const int gr = lane >> 2, tc = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        atomicAdd(reinterpret_cast<float2 *>(g + (n0 + gr) * ldg + col0 + j * 8 + tc), make_float2(acc[j][0], acc[j][1]));
        atomicAdd(reinterpret_cast<float2 *>(g + (n0 + gr + 8) * ldg + col0 + j * 8 + tc),
                  make_float2(acc[j][2], acc[j][3]));
    }
}

// column sums of a warp's 16 rows (values v[j][0..3] as in the accumulator layout), added to g
template <int NT>
__device__ __forceinline__ void atomic_add_colsum(float *g, const float (&v)[NT][4], int lane)
{
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        float s0 = v[j][0] + v[j][2], s1 = v[j][1] + v[j][3];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane < 4) atomicAdd(reinterpret_cast<float2 *>(g + j * 8 + lane * 2), make_float2(s0, s1));
    }
}

// ------------------------------------------------------------------ tile bookkeeping

struct RowMap {
    int row_race[TILE];   // race index of each row (-1: padding)
    int row_comp[TILE];   // competitor index within its race
    int row_state[TILE];  // race position within the tile
    int state_row0[MAX_STATES + 1];
    int state_n[MAX_STATES];
    int state_race[MAX_STATES];
};

__device__ void build_rowmap(RowMap &m, const SgArgs &a, const SgTile &t, int tid)
{
    if (tid < t.ns) {
        const int r = a.order[t.s0 + tid];
        m.state_race[tid] = r;
        m.state_n[tid] = a.b.race_off[r + 1] - a.b.race_off[r];
    }
    __syncthreads();
    if (tid == 0) {
        int row = 0;
        for (int i = 0; i < t.ns; ++i) {
            m.state_row0[i] = row;
            row += m.state_n[i];
        }
        m.state_row0[t.ns] = row;
    }
    if (tid < TILE) m.row_race[tid] = -1;
    __syncthreads();
    if (tid < t.ns) {
        const int r0 = m.state_row0[tid];
        for (int c = 0; c < m.state_n[tid]; ++c) {
            m.row_race[r0 + c] = m.state_race[tid];
            m.row_comp[r0 + c] = c;
            m.row_state[r0 + c] = tid;
        }
    }
    __syncthreads();
}

// Input features of every row (float32, rounded to bfloat16 into x[row][0..15]): the raw
// quantities [d/L, (L-d)/5000, mu-16, sigma-1, 2 rho-1] and, per race, the expected finish
// time T = (L-d)/v with v = mu (1 + 0.1 (2 rho - 1) d/L), its spread s = sigma sqrt(T)/v, the
// lag behind the race's least T and its z-score, the gap to the nearest competitor strictly
// ahead, and 1/n.  Called by all threads of the block.
struct FeatScratch {
    float T[TILE], sd[TILE], d[TILE], v[TILE], raw[TILE][RAW];
};

__device__ void tile_features(bf16 *x, int ldx, bf16 *ws_x, FeatScratch &fs, const SgArgs &a, const RowMap &m,
                              int tid)
{
    if (tid < TILE) {
        const int r = m.row_race[tid];
        if (r >= 0) {
            const int i = a.b.race_off[r] + m.row_comp[tid];
            const float L = a.b.L[r], d = a.b.d0[i], mu = a.b.mu[i], sigma = a.b.sigma[i], rho = a.b.rho[i];
            const float frac = d / L;
            const float v = mu * (1.0f + 0.1f * (2.0f * rho - 1.0f) * frac);
            const float T = (L - d) / v;
            fs.T[tid] = T;
            fs.v[tid] = v;
            fs.sd[tid] = sigma * sqrtf(T) / v;
            fs.d[tid] = d;
            fs.raw[tid][0] = frac;
            fs.raw[tid][1] = (L - d) / L_SCALE;
            fs.raw[tid][2] = mu - 16.0f;
            fs.raw[tid][3] = sigma - 1.0f;
            fs.raw[tid][4] = 2.0f * rho - 1.0f;
        }
    }
    __syncthreads();
    if (tid < TILE) {
        float f[KIN];
#pragma unroll
        for (int k = 0; k < KIN; ++k) f[k] = 0.0f;
        if (m.row_race[tid] >= 0) {
            const int st = m.row_state[tid];
            const int r0 = m.state_row0[st], r1 = m.state_row0[st + 1];
            int kmin = r0, ia = -1, ib = -1;
            const float dc = fs.d[tid];
            for (int q = r0; q < r1; ++q) {
                if (fs.T[q] < fs.T[kmin]) kmin = q;
                if (fs.d[q] > dc && (ia < 0 || fs.d[q] < fs.d[ia])) ia = q;
                if (fs.d[q] < dc && (ib < 0 || fs.d[q] > fs.d[ib])) ib = q;
            }
            const float ga = ia >= 0 ? fs.d[ia] - dc : 100.0f;
            const float gb = ib >= 0 ? dc - fs.d[ib] : 100.0f;
            const float gap = ga;
            const float lag = fs.T[tid] - fs.T[kmin];
            const float vc = fs.v[tid];
            f[11] = fminf(gb, 100.0f) / 10.0f;
            f[12] = (ia >= 0 && vc > fs.v[ia]) ? fminf(ga / (vc - fs.v[ia]) / fs.T[tid], 2.0f) / 2.0f : 1.0f;
            f[13] = (ib >= 0 && fs.v[ib] > vc) ? fminf(gb / (fs.v[ib] - vc) / fs.T[ib], 2.0f) / 2.0f : 1.0f;
#pragma unroll
            for (int k = 0; k < RAW; ++k) f[k] = fs.raw[tid][k];
            f[5] = fs.T[tid] / 100.0f;
            f[6] = fminf(lag, 100.0f) / 10.0f;
            f[7] = fs.sd[tid];
            f[8] = fminf(lag / sqrtf(fs.sd[tid] * fs.sd[tid] + fs.sd[kmin] * fs.sd[kmin] + 0.01f), 20.0f) / 5.0f;
            f[9] = fminf(gap, 100.0f) / 10.0f;
            f[10] = 1.0f / float(r1 - r0);
        }
#pragma unroll
        for (int k = 0; k < KIN; ++k) {
            const bf16 v = __float2bfloat16_rn(f[k]);
            x[tid * ldx + k] = v;
            if (ws_x) ws_x[tid * KIN + k] = v;
        }
    }
}

// mean over each race's rows of h (bf16, stride ldh) into g (bf16, stride ldg, per row);
// padding rows get zeros so that nothing undefined reaches a matrix product
__device__ void pool_context(bf16 *g, int ldg, const bf16 *h, int ldh, const RowMap &m, int ns, int tid)
{
    if (tid < H) {
        const int col = tid;
        for (int s = 0; s < ns; ++s) {
            const int r0 = m.state_row0[s], r1 = m.state_row0[s + 1];
            float sum = 0.0f;
            for (int row = r0; row < r1; ++row) sum += __bfloat162float(h[row * ldh + col]);
            const bf16 gv = __float2bfloat16_rn(sum / float(r1 - r0));
            for (int row = r0; row < r1; ++row) g[row * ldg + col] = gv;
        }
        for (int row = m.state_row0[ns]; row < TILE; ++row) g[row * ldg + col] = __float2bfloat16_rn(0.0f);
    }
}

// ------------------------------------------------------------------ forward

struct FwdSmem {
    bf16 w[TILE * LD_2H];
    bf16 x[TILE * LD_IN];
    bf16 ha[TILE * LD_H];
    bf16 hg[TILE * LD_2H];
    float logit[TILE];
    RowMap m;
    FeatScratch fs;
};

// bias + ReLU epilogue of a [16 x 128] warp block into shared memory (and optionally global)
template <int NT>
__device__ __forceinline__ void relu_store(float (&acc)[NT][4], const float *bias, bf16 *dst, int ld, bf16 *gdst,
                                           int row0, int lane)
{
    const int gr = lane >> 2, tc = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int col = j * 8 + tc;
        const float b0 = bias[col], b1 = bias[col + 1];
        const __nv_bfloat162 lo = __floats2bfloat162_rn(fmaxf(acc[j][0] + b0, 0.0f), fmaxf(acc[j][1] + b1, 0.0f));
        const __nv_bfloat162 hi = __floats2bfloat162_rn(fmaxf(acc[j][2] + b0, 0.0f), fmaxf(acc[j][3] + b1, 0.0f));
        *reinterpret_cast<__nv_bfloat162 *>(dst + (row0 + gr) * ld + col) = lo;
        *reinterpret_cast<__nv_bfloat162 *>(dst + (row0 + gr + 8) * ld + col) = hi;
        if (gdst) {
            *reinterpret_cast<__nv_bfloat162 *>(gdst + (row0 + gr) * H + col) = lo;
            *reinterpret_cast<__nv_bfloat162 *>(gdst + (row0 + gr + 8) * H + col) = hi;
        }
    }
}

__global__ void __launch_bounds__(NTHREADS, 1) sg_forward(SgArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem &sm = *reinterpret_cast<FwdSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = warp * 16;
    const SgTile t = a.tiles[blockIdx.x];
    build_rowmap(sm.m, a, t, tid);
    bf16 *ws = a.train ? a.ws + size_t(blockIdx.x) * (WS_X + 4 * WS_H) : nullptr;
    tile_features(sm.x, LD_IN, ws, sm.fs, a, sm.m, tid);
    load_rows<KIN>(sm.w, LD_IN, a.wb + OFF_W1, tid);
    __syncthreads();
    float acc[16][4];
    // layer 1: h1 = relu(W1 x + b1) -> ha
    zero_acc(acc);
    gemm_xwT<16, KIN>(acc, sm.x + row0 * LD_IN, LD_IN, sm.w, LD_IN, lane);
    relu_store(acc, a.wf + OFF_B1, sm.ha, LD_H, ws ? ws + WS_X : nullptr, row0, lane);
    __syncthreads();
    // layer 2: h2 = relu(W2 h1 + b2) -> hg[:, 0:128]
    load_rows<H>(sm.w, LD_H, a.wb + OFF_W2, tid);
    __syncthreads();
    zero_acc(acc);
    gemm_xwT<16, H>(acc, sm.ha + row0 * LD_H, LD_H, sm.w, LD_H, lane);
    relu_store(acc, a.wf + OFF_B2, sm.hg, LD_2H, ws ? ws + WS_X + WS_H : nullptr, row0, lane);
    __syncthreads();
    // layer 3: h3 = relu(W3 h2 + b3) -> ha
    load_rows<H>(sm.w, LD_H, a.wb + OFF_W3, tid);
    __syncthreads();
    zero_acc(acc);
    gemm_xwT<16, H>(acc, sm.hg + row0 * LD_2H, LD_2H, sm.w, LD_H, lane);
    relu_store(acc, a.wf + OFF_B3, sm.ha, LD_H, ws ? ws + WS_X + 2 * WS_H : nullptr, row0, lane);
    __syncthreads();
    // [h3 ; g] -> hg
    load_rows<2 * H>(sm.w, LD_2H, a.wb + OFF_W4, tid);
    pool_context(sm.hg + H, LD_2H, sm.ha, LD_H, sm.m, t.ns, tid);
    for (int i = tid; i < TILE * (H / 8); i += NTHREADS) {
        const int r = i / (H / 8), v = i - r * (H / 8);
        *reinterpret_cast<uint4 *>(sm.hg + r * LD_2H + v * 8) = *reinterpret_cast<const uint4 *>(sm.ha + r * LD_H + v * 8);
    }
    __syncthreads();
    // head: u = relu(W4 [h3; g] + b4); logit = w5 . bf16(u) + b5
    zero_acc(acc);
    gemm_xwT<16, 2 * H>(acc, sm.hg + row0 * LD_2H, LD_2H, sm.w, LD_2H, lane);
    {
        const int gr = lane >> 2, tc = (lane & 3) * 2;
        const float *b4 = a.wf + OFF_B4, *w5 = a.wf + OFF_W5;
        bf16 *wu = ws ? ws + WS_X + 3 * WS_H : nullptr;
        float s_lo = 0.0f, s_hi = 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = j * 8 + tc;
            const __nv_bfloat162 lo = __floats2bfloat162_rn(fmaxf(acc[j][0] + b4[col], 0.0f), fmaxf(acc[j][1] + b4[col + 1], 0.0f));
            const __nv_bfloat162 hi = __floats2bfloat162_rn(fmaxf(acc[j][2] + b4[col], 0.0f), fmaxf(acc[j][3] + b4[col + 1], 0.0f));
            s_lo += __low2float(lo) * w5[col] + __high2float(lo) * w5[col + 1];
            s_hi += __low2float(hi) * w5[col] + __high2float(hi) * w5[col + 1];
            if (wu) {
                *reinterpret_cast<__nv_bfloat162 *>(wu + (row0 + gr) * H + col) = lo;
                *reinterpret_cast<__nv_bfloat162 *>(wu + (row0 + gr + 8) * H + col) = hi;
            }
        }
        s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 1);
        s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 2);
        s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 1);
        s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 2);
        if ((lane & 3) == 0) {
            sm.logit[row0 + gr] = s_lo + a.wf[OFF_B5];
            sm.logit[row0 + gr + 8] = s_hi + a.wf[OFF_B5];
        }
    }
    __syncthreads();
    // softmax over each race's rows; training: d loss / d logit and the loss
    if (tid < t.ns) {
        const int r0 = sm.m.state_row0[tid], r1 = sm.m.state_row0[tid + 1];
        const int race = sm.m.state_race[tid];
        const int base = a.b.race_off[race];
        float mx = -INFINITY;
        for (int row = r0; row < r1; ++row) mx = fmaxf(mx, sm.logit[row]);
        float sum = 0.0f;
        for (int row = r0; row < r1; ++row) sum += expf(sm.logit[row] - mx);
        const float lsum = logf(sum);
        float tsum = 0.0f, lossv = 0.0f;
        if (a.train)
            for (int row = r0; row < r1; ++row) tsum += a.target[base + (row - r0)];
        for (int row = r0; row < r1; ++row) {
            const float lq = sm.logit[row] - mx - lsum;  // log q
            const float q = expf(lq);
            if (a.probs) a.probs[base + (row - r0)] = q;
            if (a.train) {
                const float tv = a.target[base + (row - r0)];
                a.ws_dlogit[size_t(blockIdx.x) * TILE + row] = (q * tsum - tv) * a.inv_races;
                lossv -= tv * lq;
            }
        }
        if (a.train && a.loss_acc) atomicAdd(a.loss_acc, lossv * a.inv_races);
    }
    if (a.train && tid < TILE && tid >= t.nrows) a.ws_dlogit[size_t(blockIdx.x) * TILE + tid] = 0.0f;
}

// ------------------------------------------------------------------ backward

struct BwdSmem {
    bf16 w[TILE * LD_2H];
    bf16 dy[TILE * LD_H];
    bf16 x[TILE * LD_2H];
    float dg[MAX_STATES * H];
    float dlogit[TILE];
    RowMap m;
};

// mask by (act > 0), column sums into the bias gradient, bfloat16 into dst (this warp's rows)
__device__ __forceinline__ void relu_grad_store(float (&acc)[16][4], const bf16 *act, int lda, bf16 *dst, int ldd,
                                                float *gbias, int row0, const RowMap &m, int lane)
{
    const int gr = lane >> 2, tc = (lane & 3) * 2;
    const bool lo_ok = m.row_race[row0 + gr] >= 0, hi_ok = m.row_race[row0 + gr + 8] >= 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int col = j * 8 + tc;
        const __nv_bfloat162 al = *reinterpret_cast<const __nv_bfloat162 *>(act + (row0 + gr) * lda + col);
        const __nv_bfloat162 ah = *reinterpret_cast<const __nv_bfloat162 *>(act + (row0 + gr + 8) * lda + col);
        acc[j][0] = (lo_ok && __low2float(al) > 0.0f) ? acc[j][0] : 0.0f;
        acc[j][1] = (lo_ok && __high2float(al) > 0.0f) ? acc[j][1] : 0.0f;
        acc[j][2] = (hi_ok && __low2float(ah) > 0.0f) ? acc[j][2] : 0.0f;
        acc[j][3] = (hi_ok && __high2float(ah) > 0.0f) ? acc[j][3] : 0.0f;
        *reinterpret_cast<__nv_bfloat162 *>(dst + (row0 + gr) * ldd + col) = __floats2bfloat162_rn(acc[j][0], acc[j][1]);
        *reinterpret_cast<__nv_bfloat162 *>(dst + (row0 + gr + 8) * ldd + col) = __floats2bfloat162_rn(acc[j][2], acc[j][3]);
    }
    atomic_add_colsum(gbias, acc, lane);
}

__global__ void __launch_bounds__(NTHREADS, 1) sg_backward(SgArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &sm = *reinterpret_cast<BwdSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = warp * 16;
    const SgTile t = a.tiles[blockIdx.x];
    build_rowmap(sm.m, a, t, tid);
    const bf16 *ws = a.ws + size_t(blockIdx.x) * (WS_X + 4 * WS_H);
    const bf16 *ws_x = ws, *ws_h1 = ws + WS_X, *ws_h2 = ws_h1 + WS_H, *ws_h3 = ws_h2 + WS_H, *ws_u = ws_h3 + WS_H;
    float *g = a.grad;
    if (tid < TILE) sm.dlogit[tid] = a.ws_dlogit[size_t(blockIdx.x) * TILE + tid];
    for (int i = tid; i < MAX_STATES * H; i += NTHREADS) sm.dg[i] = 0.0f;
    load_rows<H>(sm.x, LD_2H, ws_u, tid);
    __syncthreads();
    // head: du = dlogit w5 [u > 0]; d w5 = sum dlogit u; d b4 = sum du; d b5 = sum dlogit
    {
        const int col = tid & (H - 1), half = tid >> 7;
        const float w5c = a.wf[OFF_W5 + col];
        float sdu = 0.0f, sw5 = 0.0f;
        for (int row = half * 64; row < half * 64 + 64; ++row) {
            const float u = __bfloat162float(sm.x[row * LD_2H + col]);
            const float dl = sm.dlogit[row];
            const float du = u > 0.0f ? dl * w5c : 0.0f;
            sdu += du;
            sw5 += dl * u;
            sm.dy[row * LD_H + col] = __float2bfloat16_rn(du);
        }
        atomicAdd(g + OFF_B4 + col, sdu);
        atomicAdd(g + OFF_W5 + col, sw5);
        if (tid == 0) {
            float s = 0.0f;
            for (int row = 0; row < TILE; ++row) s += sm.dlogit[row];
            atomicAdd(g + OFF_B5, s);
        }
    }
    __syncthreads();
    // z = [h3 ; g] -> x
    load_rows<H>(sm.x, LD_2H, ws_h3, tid);
    __syncthreads();
    pool_context(sm.x + H, LD_2H, sm.x, LD_2H, sm.m, t.ns, tid);
    load_rows<2 * H>(sm.w, LD_2H, a.wb + OFF_W4, tid);
    __syncthreads();
    float acc[16][4];
    // d W4 = du^T z  (two halves of z's columns)
    for (int half = 0; half < 2; ++half) {
        zero_acc(acc);
        gemm_dyT_x<16>(acc, sm.dy, LD_H, row0, sm.x + half * H, LD_2H, lane);
        atomic_add_block(g + OFF_W4, 2 * H, row0, half * H, acc, lane);
    }
    // dz = du W4: the context half, summed over each race's rows
    {
        zero_acc(acc);
        gemm_dyW<16, H>(acc, sm.dy + row0 * LD_H, LD_H, sm.w + H, LD_2H, lane);
        const int gr = lane >> 2, tc = (lane & 3) * 2;
        const int rl = row0 + gr, rh = row0 + gr + 8;
        const int sl = sm.m.row_race[rl] >= 0 ? sm.m.row_state[rl] : -1;
        const int sh = sm.m.row_race[rh] >= 0 ? sm.m.row_state[rh] : -1;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = j * 8 + tc;
            if (sl >= 0) {
                atomicAdd(&sm.dg[sl * H + col], acc[j][0]);
                atomicAdd(&sm.dg[sl * H + col + 1], acc[j][1]);
            }
            if (sh >= 0) {
                atomicAdd(&sm.dg[sh * H + col], acc[j][2]);
                atomicAdd(&sm.dg[sh * H + col + 1], acc[j][3]);
            }
        }
    }
    __syncthreads();
    // the h3 half plus the pooled context's share: dh3 = dz_h3 + (1/n) sum_race dz_g, masked
    {
        zero_acc(acc);
        gemm_dyW<16, H>(acc, sm.dy + row0 * LD_H, LD_H, sm.w, LD_2H, lane);
        const int gr = lane >> 2, tc = (lane & 3) * 2;
        const int rl = row0 + gr, rh = row0 + gr + 8;
        const int sl = sm.m.row_race[rl] >= 0 ? sm.m.row_state[rl] : -1;
        const int sh = sm.m.row_race[rh] >= 0 ? sm.m.row_state[rh] : -1;
        const float il = sl >= 0 ? 1.0f / float(sm.m.state_n[sl]) : 0.0f;
        const float ih = sh >= 0 ? 1.0f / float(sm.m.state_n[sh]) : 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = j * 8 + tc;
            if (sl >= 0) {
                acc[j][0] += sm.dg[sl * H + col] * il;
                acc[j][1] += sm.dg[sl * H + col + 1] * il;
            }
            if (sh >= 0) {
                acc[j][2] += sm.dg[sh * H + col] * ih;
                acc[j][3] += sm.dg[sh * H + col + 1] * ih;
            }
        }
        __syncthreads();  // every warp has read du (dW4 above and both dz halves) before dh3 replaces it
        relu_grad_store(acc, sm.x, LD_2H, sm.dy, LD_H, g + OFF_B3, row0, sm.m, lane);
    }
    __syncthreads();
    // layers 3, 2: dW = dh^T a_prev, dh_prev = (dh W) [a_prev > 0]
    const bf16 *prev_act[2] = {ws_h2, ws_h1};
    const int offw[2] = {OFF_W3, OFF_W2};
    const int offb[2] = {OFF_B2, OFF_B1};
    for (int l = 0; l < 2; ++l) {
        load_rows<H>(sm.x, LD_2H, prev_act[l], tid);
        load_rows<H>(sm.w, LD_H, a.wb + offw[l], tid);
        __syncthreads();
        zero_acc(acc);
        gemm_dyT_x<16>(acc, sm.dy, LD_H, row0, sm.x, LD_2H, lane);
        atomic_add_block(g + offw[l], H, row0, 0, acc, lane);
        zero_acc(acc);
        gemm_dyW<16, H>(acc, sm.dy + row0 * LD_H, LD_H, sm.w, LD_H, lane);
        __syncthreads();  // every warp has read dh before it is replaced
        relu_grad_store(acc, sm.x, LD_2H, sm.dy, LD_H, g + offb[l], row0, sm.m, lane);
        __syncthreads();
    }
    // d W1 = dh1^T x
    for (int i = tid; i < TILE * (KIN / 8); i += NTHREADS) {
        const int r = i / (KIN / 8), v = i - r * (KIN / 8);
        *reinterpret_cast<uint4 *>(sm.x + r * LD_2H + v * 8) = *reinterpret_cast<const uint4 *>(ws_x + r * KIN + v * 8);
    }
    __syncthreads();
    float acc1[2][4];
    zero_acc(acc1);
    gemm_dyT_x<2>(acc1, sm.dy, LD_H, row0, sm.x, LD_2H, lane);
    atomic_add_block(g + OFF_W1, KIN, row0, 0, acc1, lane);
}

// ------------------------------------------------------------------ optimizer

__global__ void sg_adam(float *w, float *m, float *v, const float *grad, bf16 *wb, int n, float lr, float b1,
                        float b2, float eps, float wd, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void sg_to_bf16(const float *w, bf16 *wb, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void scatter_probs(const float *src, const int32_t *dst_index, float *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[dst_index[i]] = src[i];
}

#define SG_TRY(expr)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            bbe::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));            \
            return BBE_ERR_CUDA;                                                            \
        }                                                                                   \
    } while (0)

}  // namespace

// ------------------------------------------------------------------ host side

struct SgRanges {
    int32_t valid = 0;
    int32_t n_lo = 0, n_hi = 0;
    float L_lo = 0, L_hi = 0;
    float f_lo[RAW] = {}, f_hi[RAW] = {};
    float P_lo = 0, P_hi = 0, th_lo = 0, th_hi = 0;
    int32_t had_prev = 0;
};

struct bbe_surrogate {
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // float32 [N_PARAMS]
    bf16 *wb = nullptr;                                                // bfloat16 copy
    int64_t step = 0;
    // training plan state
    uint64_t epoch = 0;
    int64_t cursor = 0;                // next position in the epoch's order
    std::vector<int32_t> epoch_order;  // races of the current epoch, shuffled
    const bbe_batch *plan_batch = nullptr;
    // device scratch
    SgTile *d_tiles = nullptr;
    size_t tiles_cap = 0;
    int32_t *d_order = nullptr;
    size_t order_cap = 0;
    bf16 *ws = nullptr;
    float *ws_dlogit = nullptr;
    size_t ws_tiles = 0;
    float *d_loss = nullptr;
    SgRanges ranges;
    uint64_t ranges_version = 1;
    // inference plan cached per (batch, ranges): network races packed into tiles, fallback races
    uint64_t iplan_serial = 0, iplan_version = 0;
    std::vector<int32_t> iplan_mc;
    std::vector<uint8_t> iplan_flag;
    int64_t iplan_tiles = 0;
    SgTile *d_itiles = nullptr;
    size_t itiles_cap = 0;
    int32_t *d_iorder = nullptr;
    size_t iorder_cap = 0;
};

namespace {

size_t fwd_smem() { return sizeof(FwdSmem); }
size_t bwd_smem() { return sizeof(BwdSmem); }

bbe_status ensure_attrs()
{
    static bool done = false;
    if (done) return BBE_OK;
    SG_TRY(cudaFuncSetAttribute(sg_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(fwd_smem())));
    SG_TRY(cudaFuncSetAttribute(sg_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bwd_smem())));
    done = true;
    return BBE_OK;
}

// greedy packing of races (in the given order) into tiles of <= 128 rows and <= 64 races
void pack_tiles(const std::vector<int32_t> &off, const int32_t *order, int64_t count, int64_t base,
                std::vector<SgTile> &tiles)
{
    SgTile cur{int32_t(base), 0, 0, 0};
    for (int64_t i = 0; i < count; ++i) {
        const int r = order[i];
        const int n = off[r + 1] - off[r];
        if (cur.ns > 0 && (cur.nrows + n > TILE || cur.ns == MAX_STATES)) {
            tiles.push_back(cur);
            cur = SgTile{int32_t(base + i), 0, 0, 0};
        }
        cur.ns += 1;
        cur.nrows += n;
    }
    if (cur.ns > 0) tiles.push_back(cur);
}

template <typename T>
bbe_status ensure_buf(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return BBE_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    SG_TRY(cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T)));
    cap = need;
    return BBE_OK;
}

bbe_status ensure_ws(bbe_surrogate *s, size_t tiles)
{
    if (tiles <= s->ws_tiles && s->ws) return BBE_OK;
    if (s->ws) cudaFree(s->ws);
    if (s->ws_dlogit) cudaFree(s->ws_dlogit);
    s->ws = nullptr;
    s->ws_dlogit = nullptr;
    s->ws_tiles = 0;
    SG_TRY(cudaMalloc(&s->ws, tiles * (WS_X + 4 * WS_H) * sizeof(bf16)));
    SG_TRY(cudaMalloc(&s->ws_dlogit, tiles * TILE * sizeof(float)));
    s->ws_tiles = tiles;
    return BBE_OK;
}

SgArgs base_args(const bbe_surrogate *s, const bbe_batch *b)
{
    SgArgs a{};
    a.wb = s->wb;
    a.wf = s->w;
    a.b = b->dev;
    a.tiles = s->d_tiles;
    a.order = s->d_order;
    return a;
}

// upload order + tiles (synchronous on the stream: the host vectors are temporaries)
bbe_status upload_plan(bbe_surrogate *s, const std::vector<int32_t> &order, const std::vector<SgTile> &tiles,
                       cudaStream_t st)
{
    bbe_status e;
    if ((e = ensure_buf(s->d_order, s->order_cap, order.size()))) return e;
    if ((e = ensure_buf(s->d_tiles, s->tiles_cap, tiles.size()))) return e;
    SG_TRY(cudaMemcpyAsync(s->d_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SG_TRY(cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(SgTile), cudaMemcpyHostToDevice, st));
    SG_TRY(cudaStreamSynchronize(st));
    return BBE_OK;
}

// one training pass (forward + backward) over tiles [t0, t1) of the uploaded plan
bbe_status train_pass(bbe_surrogate *s, const bbe_batch *b, const float *target, int64_t t0, int64_t t1,
                      int64_t races, float *loss_slot, cudaStream_t st)
{
    const int64_t nt = t1 - t0;
    if (nt <= 0) return BBE_OK;
    bbe_status e;
    if ((e = ensure_ws(s, size_t(nt)))) return e;
    SgArgs a = base_args(s, b);
    a.tiles = s->d_tiles + t0;
    a.target = target;
    a.inv_races = 1.0f / float(races);
    a.loss_acc = loss_slot;
    a.grad = s->grad;
    a.ws = s->ws;
    a.ws_dlogit = s->ws_dlogit;
    a.train = 1;
    SG_TRY(cudaMemsetAsync(s->grad, 0, N_PARAMS * sizeof(float), st));
    sg_forward<<<unsigned(nt), NTHREADS, fwd_smem(), st>>>(a);
    SG_TRY(cudaGetLastError());
    sg_backward<<<unsigned(nt), NTHREADS, bwd_smem(), st>>>(a);
    SG_TRY(cudaGetLastError());
    return BBE_OK;
}

float feature(int k, float d, float L, float mu, float sigma, float rho)
{
    switch (k) {
    case 0: return d / L;
    case 1: return (L - d) / L_SCALE;
    case 2: return mu - 16.0f;
    case 3: return sigma - 1.0f;
    default: return 2.0f * rho - 1.0f;
    }
}

void record_ranges(SgRanges &R, const bbe_batch *b)
{
    R = SgRanges{};
    R.valid = 1;
    R.n_lo = 1 << 30;
    R.n_hi = 0;
    R.L_lo = R.P_lo = R.th_lo = INFINITY;
    R.L_hi = R.P_hi = R.th_hi = -INFINITY;
    for (int k = 0; k < RAW; ++k) {
        R.f_lo[k] = INFINITY;
        R.f_hi[k] = -INFINITY;
    }
    R.had_prev = b->h_prev.empty() ? 0 : 1;
    for (int r = 0; r < b->n_races; ++r) {
        const int n = b->h_off[r + 1] - b->h_off[r];
        R.n_lo = std::min(R.n_lo, n);
        R.n_hi = std::max(R.n_hi, n);
        const float L = b->h_L[r];
        R.L_lo = std::min(R.L_lo, L);
        R.L_hi = std::max(R.L_hi, L);
        for (int i = b->h_off[r]; i < b->h_off[r + 1]; ++i) {
            for (int k = 0; k < RAW; ++k) {
                const float f = feature(k, b->h_d0[i], L, b->h_mu[i], b->h_sigma[i], b->h_rho[i]);
                R.f_lo[k] = std::min(R.f_lo[k], f);
                R.f_hi[k] = std::max(R.f_hi[k], f);
            }
            R.P_lo = std::min(R.P_lo, b->h_P[i]);
            R.P_hi = std::max(R.P_hi, b->h_P[i]);
            R.th_lo = std::min(R.th_lo, b->h_theta[i]);
            R.th_hi = std::max(R.th_hi, b->h_theta[i]);
        }
    }
}

bool in_range(const SgRanges &R, const bbe_batch *b, int r)
{
    const int n = b->h_off[r + 1] - b->h_off[r];
    if (n < R.n_lo || n > R.n_hi) return false;
    const float L = b->h_L[r];
    if (!(L >= R.L_lo && L <= R.L_hi)) return false;
    if (!b->h_prev.empty() && !R.had_prev) return false;
    for (int i = b->h_off[r]; i < b->h_off[r + 1]; ++i) {
        for (int k = 0; k < RAW; ++k) {
            const float f = feature(k, b->h_d0[i], L, b->h_mu[i], b->h_sigma[i], b->h_rho[i]);
            if (!(f >= R.f_lo[k] && f <= R.f_hi[k])) return false;
        }
        if (!(b->h_P[i] >= R.P_lo && b->h_P[i] <= R.P_hi)) return false;
        if (!(b->h_theta[i] >= R.th_lo && b->h_theta[i] <= R.th_hi)) return false;
    }
    return true;
}

// splitmix64-driven uniform in [-1, 1)
struct InitRng {
    uint64_t x;
    double next()
    {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return double(z >> 11) * 0x1.0p-52 - 1.0;
    }
};

bbe_status alloc_surrogate(bbe_surrogate *s)
{
    SG_TRY(cudaMalloc(&s->w, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMalloc(&s->m, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMalloc(&s->v, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMalloc(&s->grad, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMalloc(&s->wb, N_PARAMS * sizeof(bf16)));
    SG_TRY(cudaMalloc(&s->d_loss, sizeof(float)));
    SG_TRY(cudaMemset(s->m, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMemset(s->v, 0, N_PARAMS * sizeof(float)));
    return BBE_OK;
}

bbe_status upload_params(bbe_surrogate *s, const float *host)
{
    SG_TRY(cudaMemcpy(s->w, host, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    sg_to_bf16<<<(N_PARAMS + 255) / 256, 256>>>(s->w, s->wb, N_PARAMS);
    SG_TRY(cudaGetLastError());
    SG_TRY(cudaMemset(s->m, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMemset(s->v, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaDeviceSynchronize());
    s->step = 0;
    return BBE_OK;
}

void free_surrogate(bbe_surrogate *s)
{
    for (void *p : {(void *)s->w, (void *)s->m, (void *)s->v, (void *)s->grad, (void *)s->wb, (void *)s->d_tiles,
                    (void *)s->d_order, (void *)s->ws, (void *)s->ws_dlogit, (void *)s->d_loss, (void *)s->d_itiles,
                    (void *)s->d_iorder})
        if (p) cudaFree(p);
}

// forward over all races of b in batch order (no range check)
bbe_status forward_all(bbe_surrogate *s, const bbe_batch *b, const std::vector<int32_t> &order, float *probs,
                       cudaStream_t st)
{
    if (order.empty()) return BBE_OK;
    std::vector<SgTile> tiles;
    pack_tiles(b->h_off, order.data(), int64_t(order.size()), 0, tiles);
    bbe_status e;
    if ((e = ensure_attrs())) return e;
    if ((e = upload_plan(s, order, tiles, st))) return e;
    SgArgs a = base_args(s, b);
    a.probs = probs;
    a.train = 0;
    sg_forward<<<unsigned(tiles.size()), NTHREADS, fwd_smem(), st>>>(a);
    SG_TRY(cudaGetLastError());
    return BBE_OK;
}

}  // namespace

extern "C" {

int64_t bbe_surrogate_num_params(void) { return N_PARAMS; }

bbe_status bbe_surrogate_create(bbe_surrogate **out, uint64_t init_seed)
{
    if (!out) {
        bbe::set_error("out is NULL");
        return BBE_ERR_ARG;
    }
    *out = nullptr;
    auto s = new bbe_surrogate();
    bbe_status e = alloc_surrogate(s);
    if (e) {
        free_surrogate(s);
        delete s;
        return e;
    }
    std::vector<float> p(N_PARAMS, 0.0f);
    InitRng rng{init_seed};
    auto fill = [&](int off, int rows, int cols, int fan_in, int used_cols, double gain) {
        const double bound = std::sqrt(gain / fan_in);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) p[off + r * cols + c] = c < used_cols ? float(rng.next() * bound) : 0.0f;
    };
    fill(OFF_W1, H, KIN, FIN, FIN, 6.0);
    fill(OFF_W2, H, H, H, H, 6.0);
    fill(OFF_W3, H, H, H, H, 6.0);
    fill(OFF_W4, H, 2 * H, 2 * H, 2 * H, 6.0);
    fill(OFF_W5, 1, H, H, H, 3.0);
    if ((e = upload_params(s, p.data()))) {
        free_surrogate(s);
        delete s;
        return e;
    }
    *out = s;
    return BBE_OK;
}

bbe_status bbe_surrogate_set_params(bbe_surrogate *s, const float *params)
{
    if (!s || !params) {
        bbe::set_error("surrogate or params is NULL");
        return BBE_ERR_ARG;
    }
    return upload_params(s, params);
}

bbe_status bbe_surrogate_get_params(const bbe_surrogate *s, float *params)
{
    if (!s || !params) {
        bbe::set_error("surrogate or params is NULL");
        return BBE_ERR_ARG;
    }
    SG_TRY(cudaDeviceSynchronize());
    SG_TRY(cudaMemcpy(params, s->w, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return BBE_OK;
}

bbe_status bbe_surrogate_grad(bbe_surrogate *s, const bbe_batch *b, const float *target, float *grad, float *loss,
                              void *cuda_stream)
{
    if (!s || !b || !target || !grad) {
        bbe::set_error("surrogate, batch, target or grad is NULL");
        return BBE_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    bbe_status e;
    if ((e = ensure_attrs())) return e;
    std::vector<int32_t> order(b->n_races);
    std::iota(order.begin(), order.end(), 0);
    std::vector<SgTile> tiles;
    pack_tiles(b->h_off, order.data(), int64_t(order.size()), 0, tiles);
    if ((e = upload_plan(s, order, tiles, st))) return e;
    if (loss) SG_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    if ((e = train_pass(s, b, target, 0, int64_t(tiles.size()), b->n_races, loss, st))) return e;
    SG_TRY(cudaMemcpyAsync(grad, s->grad, N_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return BBE_OK;
}

bbe_status bbe_surrogate_train(bbe_surrogate *s, const bbe_batch *b, const float *target, const bbe_train_cfg *cfg,
                               float *loss_log, void *cuda_stream)
{
    if (!s || !b || !target || !cfg || cfg->batch_states < 1 || cfg->steps < 1 || !(cfg->lr > 0.0f) ||
        !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps > 0.0f) || !(cfg->weight_decay >= 0.0f)) {
        bbe::set_error("bbe_surrogate_train: bad arguments");
        return BBE_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    bbe_status e;
    if ((e = ensure_attrs())) return e;
    if (!s->ranges.valid) {
        record_ranges(s->ranges, b);
        s->ranges_version += 1;
    }
    if (s->plan_batch != b || int64_t(s->epoch_order.size()) != b->n_races) {
        s->plan_batch = b;
        s->epoch_order.clear();
        s->cursor = 0;
    }
    if (loss_log) SG_TRY(cudaMemsetAsync(loss_log, 0, size_t(cfg->steps) * sizeof(float), st));
    for (int32_t k = 0; k < cfg->steps; ++k) {
        if (s->epoch_order.empty() || s->cursor >= int64_t(s->epoch_order.size())) {
            s->epoch_order.resize(b->n_races);
            std::iota(s->epoch_order.begin(), s->epoch_order.end(), 0);
            std::mt19937_64 rng(cfg->shuffle_seed ^ (0x9E3779B97F4A7C15ull * (s->epoch + 1)));
            std::shuffle(s->epoch_order.begin(), s->epoch_order.end(), rng);
            s->epoch += 1;
            s->cursor = 0;
        }
        const int64_t take = std::min<int64_t>(cfg->batch_states, int64_t(s->epoch_order.size()) - s->cursor);
        std::vector<int32_t> order(s->epoch_order.begin() + s->cursor, s->epoch_order.begin() + s->cursor + take);
        s->cursor += take;
        std::vector<SgTile> tiles;
        pack_tiles(b->h_off, order.data(), take, 0, tiles);
        if ((e = upload_plan(s, order, tiles, st))) return e;
        if ((e = train_pass(s, b, target, 0, int64_t(tiles.size()), take, loss_log ? loss_log + k : nullptr, st)))
            return e;
        s->step += 1;
        const float c1 = 1.0f - std::pow(cfg->beta1, float(s->step));
        const float c2 = 1.0f - std::pow(cfg->beta2, float(s->step));
        sg_adam<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(s->w, s->m, s->v, s->grad, s->wb, N_PARAMS, cfg->lr,
                                                       cfg->beta1, cfg->beta2, cfg->eps, cfg->weight_decay, c1, c2);
        SG_TRY(cudaGetLastError());
    }
    return BBE_OK;
}

bbe_status bbe_surrogate_forward(bbe_surrogate *s, const bbe_batch *b, float *probs, void *cuda_stream)
{
    if (!s || !b || !probs) {
        bbe::set_error("surrogate, batch or probs is NULL");
        return BBE_ERR_ARG;
    }
    std::vector<int32_t> order(b->n_races);
    std::iota(order.begin(), order.end(), 0);
    return forward_all(s, b, order, probs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

bbe_status bbe_surrogate_infer(bbe_surrogate *s, const bbe_batch *b, float *probs, uint8_t *used_mc,
                               void *cuda_stream)
{
    if (!s || !b || !probs) {
        bbe::set_error("surrogate, batch or probs is NULL");
        return BBE_ERR_ARG;
    }
    if (!s->ranges.valid) {
        bbe::set_error("bbe_surrogate_infer: the network has no training ranges (train or load it first)");
        return BBE_ERR_RANGE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    bbe_status e;
    if ((e = ensure_attrs())) return e;
    if (s->iplan_serial != b->serial || s->iplan_version != s->ranges_version) {
        // range check and tile packing on the host, once per (batch, ranges)
        std::vector<int32_t> net;
        s->iplan_mc.clear();
        s->iplan_flag.assign(b->n_races, 0);
        for (int r = 0; r < b->n_races; ++r) {
            if (in_range(s->ranges, b, r)) {
                net.push_back(r);
            } else {
                s->iplan_mc.push_back(r);
                s->iplan_flag[r] = 1;
            }
        }
        std::vector<SgTile> tiles;
        pack_tiles(b->h_off, net.data(), int64_t(net.size()), 0, tiles);
        if ((e = ensure_buf(s->d_iorder, s->iorder_cap, net.size()))) return e;
        if ((e = ensure_buf(s->d_itiles, s->itiles_cap, tiles.size()))) return e;
        SG_TRY(cudaMemcpyAsync(s->d_iorder, net.data(), net.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        SG_TRY(cudaMemcpyAsync(s->d_itiles, tiles.data(), tiles.size() * sizeof(SgTile), cudaMemcpyHostToDevice, st));
        SG_TRY(cudaStreamSynchronize(st));
        s->iplan_tiles = int64_t(tiles.size());
        s->iplan_serial = b->serial;
        s->iplan_version = s->ranges_version;
    }
    if (s->iplan_tiles > 0) {
        SgArgs a = base_args(s, b);
        a.tiles = s->d_itiles;
        a.order = s->d_iorder;
        a.probs = probs;
        a.train = 0;
        sg_forward<<<unsigned(s->iplan_tiles), NTHREADS, fwd_smem(), st>>>(a);
        SG_TRY(cudaGetLastError());
    }
    const std::vector<int32_t> &mc = s->iplan_mc;
    const std::vector<uint8_t> &flag = s->iplan_flag;
    if (!mc.empty()) {
        // plain Monte Carlo for the out-of-range races, with their own stream ids
        std::vector<int32_t> off(1, 0), ids;
        std::vector<float> L, d0, mu, sg, rho, P, th, pv;
        std::vector<int64_t> R;
        std::vector<int32_t> dst;
        for (int r : mc) {
            const int a0 = b->h_off[r], a1 = b->h_off[r + 1];
            off.push_back(off.back() + (a1 - a0));
            L.push_back(b->h_L[r]);
            R.push_back(b->h_R[r]);
            ids.push_back(b->h_race_ids.empty() ? int32_t(b->race_id0 + uint32_t(r)) : b->h_race_ids[r]);
            for (int i = a0; i < a1; ++i) {
                d0.push_back(b->h_d0[i]);
                mu.push_back(b->h_mu[i]);
                sg.push_back(b->h_sigma[i]);
                rho.push_back(b->h_rho[i]);
                P.push_back(b->h_P[i]);
                th.push_back(b->h_theta[i]);
                if (!b->h_prev.empty()) pv.push_back(b->h_prev[i]);
                dst.push_back(i);
            }
        }
        bbe_batch *sub = nullptr;
        e = bbe::stage_batch(&sub, int32_t(mc.size()), off.data(), L.data(), R.data(), d0.data(), mu.data(), sg.data(),
                             rho.data(), P.data(), th.data(), pv.empty() ? nullptr : pv.data(), b->seed,
                             bbe_dist(b->dist), 0, ids.data(), st);
        if (e) return e;
        if ((e = bbe_batch_set_cfg(sub, &b->cfg))) {
            bbe_destroy_batch(sub);
            return e;
        }
        int32_t *counts = nullptr, *d_dst = nullptr;
        float *sub_probs = nullptr;
        const size_t nc = dst.size();
        cudaError_t ce = cudaMalloc(&counts, nc * sizeof(int32_t));
        if (ce == cudaSuccess) ce = cudaMalloc(&sub_probs, nc * sizeof(float));
        if (ce == cudaSuccess) ce = cudaMalloc(&d_dst, nc * sizeof(int32_t));
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_dst, dst.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess) {
            e = bbe_rollout_batch(sub, counts, nullptr, st);
            if (!e) e = bbe_win_probs(sub, counts, sub_probs, nullptr, st);
            if (!e) {
                scatter_probs<<<unsigned((nc + 255) / 256), 256, 0, st>>>(sub_probs, d_dst, probs, int(nc));
                ce = cudaGetLastError();
            }
            if (!e && ce == cudaSuccess) e = bbe_batch_status(sub, st);  // synchronises the stream
        }
        if (ce != cudaSuccess) {
            bbe::set_error(std::string("Monte Carlo fallback: ") + cudaGetErrorString(ce));
            e = BBE_ERR_CUDA;
        }
        cudaStreamSynchronize(st);
        cudaFree(counts);
        cudaFree(sub_probs);
        cudaFree(d_dst);
        bbe_destroy_batch(sub);
        if (e) return e;
    }
    if (used_mc) {
        SG_TRY(cudaMemcpyAsync(used_mc, flag.data(), flag.size(), cudaMemcpyHostToDevice, st));
        SG_TRY(cudaStreamSynchronize(st));
    }
    return BBE_OK;
}

bbe_status bbe_surrogate_save(const bbe_surrogate *s, const char *path)
{
    if (!s || !path) {
        bbe::set_error("surrogate or path is NULL");
        return BBE_ERR_ARG;
    }
    std::vector<float> w(N_PARAMS), m(N_PARAMS), v(N_PARAMS);
    SG_TRY(cudaDeviceSynchronize());
    SG_TRY(cudaMemcpy(w.data(), s->w, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    SG_TRY(cudaMemcpy(m.data(), s->m, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    SG_TRY(cudaMemcpy(v.data(), s->v, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) {
        bbe::set_error(std::string("cannot open ") + path);
        return BBE_ERR_ARG;
    }
    const char magic[8] = {'B', 'B', 'E', 'S', 'G', '0', '0', '1'};
    const int64_t n = N_PARAMS;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
              std::fwrite(&s->step, 8, 1, f) == 1 && std::fwrite(&s->epoch, 8, 1, f) == 1 &&
              std::fwrite(&s->cursor, 8, 1, f) == 1 && std::fwrite(&s->ranges, sizeof(SgRanges), 1, f) == 1 &&
              std::fwrite(w.data(), 4, n, f) == size_t(n) && std::fwrite(m.data(), 4, n, f) == size_t(n) &&
              std::fwrite(v.data(), 4, n, f) == size_t(n);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) {
        bbe::set_error(std::string("write failed: ") + path);
        return BBE_ERR_ARG;
    }
    return BBE_OK;
}

bbe_status bbe_surrogate_load(bbe_surrogate **out, const char *path)
{
    if (!out || !path) {
        bbe::set_error("out or path is NULL");
        return BBE_ERR_ARG;
    }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) {
        bbe::set_error(std::string("cannot open ") + path);
        return BBE_ERR_ARG;
    }
    char magic[8];
    int64_t n = 0, step = 0, cursor = 0;
    uint64_t epoch = 0;
    SgRanges ranges;
    std::vector<float> w(N_PARAMS), m(N_PARAMS), v(N_PARAMS);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "BBESG001", 8) == 0 &&
              std::fread(&n, 8, 1, f) == 1 && n == N_PARAMS && std::fread(&step, 8, 1, f) == 1 &&
              std::fread(&epoch, 8, 1, f) == 1 && std::fread(&cursor, 8, 1, f) == 1 &&
              std::fread(&ranges, sizeof(SgRanges), 1, f) == 1 && std::fread(w.data(), 4, n, f) == size_t(n) &&
              std::fread(m.data(), 4, n, f) == size_t(n) && std::fread(v.data(), 4, n, f) == size_t(n);
    std::fclose(f);
    if (!ok) {
        bbe::set_error(std::string("not a surrogate checkpoint: ") + path);
        return BBE_ERR_ARG;
    }
    auto s = new bbe_surrogate();
    bbe_status e = alloc_surrogate(s);
    if (!e) e = upload_params(s, w.data());
    if (!e) {
        cudaError_t ce = cudaMemcpy(s->m, m.data(), N_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(s->v, v.data(), N_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            bbe::set_error(std::string("checkpoint upload: ") + cudaGetErrorString(ce));
            e = BBE_ERR_CUDA;
        }
    }
    if (e) {
        free_surrogate(s);
        delete s;
        return e;
    }
    s->step = step;
    s->epoch = epoch;
    s->cursor = cursor;
    s->ranges = ranges;
    s->ranges_version += 1;
    *out = s;
    return BBE_OK;
}

void bbe_surrogate_destroy(bbe_surrogate *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    free_surrogate(s);
    delete s;
}

}  // extern "C"
