// bbe_surrogate.cu -- the win-probability surrogate network (include/bbe_surrogate.h):
// forward, backward and Adam kernels and the C ABI around them.
//
// Work is cut into tiles of at most 128 competitor rows holding whole races (at most 64),
// so that the mean-pooled context and the per-race softmax stay inside one tile.
//   forward   Y[rows][out] = X[rows][in] . W[out][in]^T on the fifth-generation tensor cores
//             (tcgen05.mma, bfloat16 operands in shared memory, float32 accumulators in
//             tensor memory), persistent blocks with the weights resident (sg_forward_tc).
//   backward  dX = dY . W per tile (sg_backward_chain) and dW = dY^T . X accumulated over
//             tiles in tensor memory, split over blocks and reduced in a fixed order
//             (sg_backward_wgrad, sg_reduce_grad), also on tcgen05.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
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

// bfloat16 image of W1..W4 in the canonical K-major operand layout of the tensor-core
// descriptors (element offsets); kept in step with the float32 parameters by the optimizer
constexpr int WC_W1 = 0;
constexpr int WC_W2 = WC_W1 + H * KIN;
constexpr int WC_W3 = WC_W2 + H * H;
constexpr int WC_W4 = WC_W3 + H * H;
constexpr int WC_ELEMS = WC_W4 + H * 2 * H;

constexpr int TC_THREADS = 512;                  // forward: two tile pipelines of two warpgroups each
constexpr int TC_PIPE = 256;                     // threads of one pipeline
constexpr long long kWaitNs = 2000000000LL;      // limit of every device-side wait (2 s)

// Training workspace of one tile (global memory, bytes).  Every [128][128] bfloat16 block is in
// the canonical activation layout (8-row x 16-byte core matrices, row-group stride 2048 B), so
// the backward kernels move each block with one bulk copy and read it as a tensor-core operand.
constexpr size_t WS_BLOCK = size_t(TILE) * H * 2;           // 32 KB
constexpr size_t WS_MASK = size_t(TILE) * (H / 32) * 4;      // 2 KB: ReLU mask bits, [row][4 words]
constexpr size_t WS_H1 = 0;                                  // h1, h2, h3, g, u
constexpr size_t WS_U = 4 * WS_BLOCK;
constexpr size_t WS_G = 3 * WS_BLOCK;
constexpr size_t WS_M = 5 * WS_BLOCK;                        // masks of h1, h2, h3, u (> 0)
constexpr size_t WS_DU = WS_M + 4 * WS_MASK;                 // du, da3, da2, da1 (backward)
constexpr size_t WS_DA3 = WS_DU + WS_BLOCK;
constexpr size_t WS_DA2 = WS_DA3 + WS_BLOCK;
constexpr size_t WS_DA1 = WS_DA2 + WS_BLOCK;
constexpr size_t WS_TILE = WS_DA1 + WS_BLOCK;                // 303,104 bytes

struct SgTile {
    int32_t s0;     // first position in the order array
    int32_t ns;     // races in the tile
    int32_t nrows;  // competitor rows
    int32_t pad;
};

// race layout of a tile, written by the feature kernel and moved into the tensor-core
// kernel by a bulk copy (size a multiple of 16 bytes)
struct TileMeta {
    int32_t ns, nrows;
    int32_t state_row0[MAX_STATES + 1];  // first row of each race; [ns] = rows in use
    int32_t state_race[MAX_STATES];      // race index of each race slot
    int8_t row_state[TILE];              // race slot of each row (-1: padding)
    int32_t pad;
};

struct SgArgs {
    const bf16 *wb;        // bfloat16 copy of the parameters (flat layout)
    const bf16 *wc;        // bfloat16 W1..W4 in the canonical operand layout (WC_*)
    const float *wf;       // float32 master parameters (biases and w5 are read from here)
    const SgTile *tiles;
    const int32_t *order;  // race indices in tile order
    bbe::DevBatch b;
    float *probs;          // forward output per competitor (batch order) or null
    const float *target;   // training targets per competitor (batch order)
    float inv_races;       // 1 / races in the step
    float *loss_acc;       // training: mean loss accumulator (device scalar) or null
    float *grad;           // training: float32 gradient (flat layout)
    unsigned char *ws;     // training workspace, WS_TILE bytes per tile
    float *partial;        // backward: per-block weight-gradient partials [2][groups][N_PARAMS]
    int32_t wgroups;       // backward: blocks per weight-gradient group
    float *ws_dlogit;      // training: d loss / d logit per tile row
    int train;
    unsigned char *xbuf;   // forward: per-tile features, canonical operand layout (TILE * KIN bf16)
    TileMeta *meta;        // forward: per-tile race layout
    float *logits;         // forward: per-tile-row logits
    int *status;           // set to 1 when a bounded device wait gave up
    long long wait_ns;     // limit of each wait
    int32_t raw_only;      // 1: the five raw inputs only (the derived columns are zero)
    float *b5_part;        // training: per tile, the sum of its d loss / d logit (the b5 gradient's terms)
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ------------------------------------------------------------------ tile bookkeeping

// barrier of the threads that work on one tile: the whole block, or the threads of one
// forward tile pipeline (named barrier 1 + pipeline)
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
    int id, count;
    __device__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory"); }
};

struct RowMap {
    int row_race[TILE];   // race index of each row (-1: padding)
    int row_comp[TILE];   // competitor index within its race
    int row_state[TILE];  // race position within the tile
    int state_row0[MAX_STATES + 1];
    int state_n[MAX_STATES];
    int state_race[MAX_STATES];
};

// called by the tile's threads (tid 0..127 at least)
template <typename Sync>
__device__ void build_rowmap(RowMap &m, const SgArgs &a, const SgTile &t, int tid, Sync sync)
{
    if (tid < t.ns) {
        const int r = a.order[t.s0 + tid];
        m.state_race[tid] = r;
        m.state_n[tid] = a.b.race_off[r + 1] - a.b.race_off[r];
    }
    sync();
    if (tid == 0) {
        int row = 0;
        for (int i = 0; i < t.ns; ++i) {
            m.state_row0[i] = row;
            row += m.state_n[i];
        }
        m.state_row0[t.ns] = row;
    }
    if (tid < TILE) m.row_race[tid] = -1;
    sync();
    if (tid < t.ns) {
        const int r0 = m.state_row0[tid];
        for (int c = 0; c < m.state_n[tid]; ++c) {
            m.row_race[r0 + c] = m.state_race[tid];
            m.row_comp[r0 + c] = c;
            m.row_state[r0 + c] = tid;
        }
    }
    sync();
}

// Input features of tile row `tid` (float32; zeros for padding rows and for tid >= 128): the
// raw quantities [d/L, (L-d)/5000, mu-16, sigma-1, 2 rho-1] and, per race, the expected finish
// time T = (L-d)/v with v = mu (1 + 0.1 (2 rho - 1) d/L), its spread s = sigma sqrt(T)/v, the
// lag behind the race's least T and its z-score, the gaps to the nearest competitors strictly
// ahead and behind, 1/n, and the catch-up shares.  Called by all threads of the tile.
struct FeatScratch {
    float T[TILE], sd[TILE], d[TILE], v[TILE], raw[TILE][RAW];
};

template <typename Sync>
__device__ void tile_features(float (&f)[KIN], FeatScratch &fs, const SgArgs &a, const RowMap &m, int tid, Sync sync)
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
    sync();
#pragma unroll
    for (int k = 0; k < KIN; ++k) f[k] = 0.0f;
    if (tid < TILE && m.row_race[tid] >= 0) {
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
        const float lag = fs.T[tid] - fs.T[kmin];
        const float vc = fs.v[tid];
#pragma unroll
        for (int k = 0; k < RAW; ++k) f[k] = fs.raw[tid][k];
        f[5] = fs.T[tid] / 100.0f;
        f[6] = fminf(lag, 100.0f) / 10.0f;
        f[7] = fs.sd[tid];
        f[8] = fminf(lag / sqrtf(fs.sd[tid] * fs.sd[tid] + fs.sd[kmin] * fs.sd[kmin] + 0.01f), 20.0f) / 5.0f;
        f[9] = fminf(ga, 100.0f) / 10.0f;
        f[10] = 1.0f / float(r1 - r0);
        f[11] = fminf(gb, 100.0f) / 10.0f;
        f[12] = (ia >= 0 && vc > fs.v[ia]) ? fminf(ga / (vc - fs.v[ia]) / fs.T[tid], 2.0f) / 2.0f : 1.0f;
        f[13] = (ib >= 0 && fs.v[ib] > vc) ? fminf(gb / (fs.v[ib] - vc) / fs.T[ib], 2.0f) / 2.0f : 1.0f;
    }
}

// ------------------------------------------------------------------ forward (tcgen05)
//
// Three launches.  sg_prep (one 128-thread block per tile, many blocks per SM so that the
// scattered loads of the race data overlap) writes each tile's bfloat16 features in the
// canonical operand layout and a record of its race layout.  sg_forward_tc is persistent:
// a block of two warpgroups runs two independent tile pipelines that share one copy of the
// layer weights, kept in shared memory for the whole launch in the canonical K-major
// operand layout (8-row x 16-byte core matrices, no swizzle); the optimizer keeps a
// bfloat16 image of W1..W4 in that layout in global memory, so four bulk asynchronous
// copies bring them in, and each tile's features and layout record arrive the same way,
// double-buffered one tile ahead.  Per layer, one thread of the warpgroup issues
// tcgen05.mma (M = 128 tile rows, N = 128 outputs, K = 16 per instruction) into the
// pipeline's 128 tensor-memory columns and commits to the pipeline's mbarrier; then the
// four warps read the float32 accumulators back (warp w of the group reads TMEM lanes
// 32w..32w+31, one tile row per thread), add the bias, apply ReLU and write bfloat16
// activations over the layer's input, which the finished product no longer reads.  The
// head [h3 ; g] W4^T is two accumulating products: h3 against the first 128 columns of W4,
// then, once the per-race mean g has replaced h3 in place, g against the other 128.  While
// one pipeline waits for its product the other one runs its epilogue on the CUDA cores.
// sg_softmax (one warp per tile) turns the logits into per-race probabilities and, when
// training, the loss and its gradient with respect to the logits.

// byte offset of element (row, k) of a canonical K-major operand with kdim columns
__host__ __device__ constexpr uint32_t canon_off(int row, int k, int kdim)
{
    return uint32_t(((row >> 3) * (kdim >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait until phase `parity` of the mbarrier has completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long limit_ns)
{
    const uint32_t addr = smem_addr(bar);
    const long long t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
    }
}

// bulk asynchronous copy global -> shared (16-byte aligned, size a multiple of 16), completing
// on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor of a canonical K-major operand without swizzle: start
// address, byte distance to the next core matrix along K (lbo) and along M or N (sbo), and
// the fixed descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// instruction descriptor of kind::f16: float32 D, bfloat16 A and B, A K-major, N = 128,
// M = 128; B K-major (kIdesc) or MN-major (kIdescBmn, bit 16).  For an MN-major operand without
// swizzle the descriptor's lbo is the byte distance between core matrices along K and sbo
// the distance along N.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(H >> 3) << 17) | (uint32_t(TILE >> 4) << 24);
constexpr uint32_t kIdescBmn = kIdesc | (1u << 16);

// D (+)= A . B^T with A and B in shared memory
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// D (+)= A . B^T with A in tensor memory (lane = row, 8 columns of bfloat16 pairs per K = 16,
// even k in the low half) and B in shared memory
__device__ __forceinline__ void tc_mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive float32 columns of this thread's TMEM lane into r[O..O+15]
template <int O, int N>
__device__ __forceinline__ void tmem_ld16(uint32_t (&r)[N], uint32_t taddr)
{
    static_assert(O + 16 <= N, "register range");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[O + 0]), "=r"(r[O + 1]), "=r"(r[O + 2]), "=r"(r[O + 3]), "=r"(r[O + 4]), "=r"(r[O + 5]),
          "=r"(r[O + 6]), "=r"(r[O + 7]), "=r"(r[O + 8]), "=r"(r[O + 9]), "=r"(r[O + 10]), "=r"(r[O + 11]),
          "=r"(r[O + 12]), "=r"(r[O + 13]), "=r"(r[O + 14]), "=r"(r[O + 15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// r[O..O+15] into 16 consecutive 32-bit columns of this thread's TMEM lane
template <int O, int N>
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[N])
{
    static_assert(O + 16 <= N, "register range");
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[O + 0]), "r"(r[O + 1]), "r"(r[O + 2]), "r"(r[O + 3]), "r"(r[O + 4]), "r"(r[O + 5]), "r"(r[O + 6]),
        "r"(r[O + 7]), "r"(r[O + 8]), "r"(r[O + 9]), "r"(r[O + 10]), "r"(r[O + 11]), "r"(r[O + 12]), "r"(r[O + 13]),
        "r"(r[O + 14]), "r"(r[O + 15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// bfloat16 pair {relu(lo), relu(hi)} rounded to nearest (lo in the low half)
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Epilogues.  Two threads share a tile row (its TMEM lane): thread half ch handles the 64
// accumulator columns [64 ch, 64 ch + 64).  In training the activations also go to the
// workspace block (same canonical offsets) and their ReLU masks (bit c mod 32 of word c / 32 of
// the row: activation c > 0) to the mask block.

// byte offset of row `row` in a canonical [128][128] activation block; chunk c (8 columns) is at
// + c * 128
__device__ __forceinline__ uint32_t act_row(int row) { return uint32_t((row >> 3) * 2048 + (row & 7) * 16); }

// mask bits of a bfloat16 pair from cvt.rn.relu (the values are +0 or positive)
__device__ __forceinline__ uint32_t pos_bits(uint32_t pk)
{
    return ((pk & 0xFFFFu) != 0u ? 1u : 0u) | ((pk >> 16) != 0u ? 2u : 0u);
}

// bias + ReLU -> bfloat16 into the canonical activation tile (and, TRAIN, the workspace block and mask)
template <bool TRAIN>
__device__ __forceinline__ void tc_epilogue_relu(uint32_t taddr, const float *bias, unsigned char *act, int row,
                                                 unsigned char *ws_blk, uint32_t *ws_mask, int c0)
{
    unsigned char *arow = act + act_row(row);
#pragma unroll
    for (int cb = c0; cb < c0 + 64; cb += 32) {
        uint32_t r[32];
        tmem_ld16<0>(r, taddr + cb);
        tmem_ld16<16>(r, taddr + cb + 16);
        tmem_wait_ld();
        uint32_t bits = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = q * 8 + 2 * e;
                pk[e] = relu_bf16x2(__uint_as_float(r[j]) + bias[cb + j], __uint_as_float(r[j + 1]) + bias[cb + j + 1]);
                if (TRAIN) bits |= pos_bits(pk[e]) << j;
            }
            const uint4 v = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4 *>(arow + ((cb >> 3) + q) * 128) = v;
            if (TRAIN) *reinterpret_cast<uint4 *>(ws_blk + act_row(row) + ((cb >> 3) + q) * 128) = v;
        }
        if (TRAIN) ws_mask[row * 4 + (cb >> 5)] = bits;
    }
}

// head: u = bfloat16(relu(acc + b4)) (workspace block and mask when training); returns this
// half's w5 . u
template <bool TRAIN>
__device__ __forceinline__ float tc_epilogue_head(uint32_t taddr, const float *b4, const float *w5, int row,
                                                  unsigned char *ws_blk, uint32_t *ws_mask, int c0)
{
    float s = 0.0f;
#pragma unroll
    for (int cb = c0; cb < c0 + 64; cb += 32) {
        uint32_t r[32];
        tmem_ld16<0>(r, taddr + cb);
        tmem_ld16<16>(r, taddr + cb + 16);
        tmem_wait_ld();
        uint32_t bits = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = q * 8 + 2 * e;
                pk[e] = relu_bf16x2(__uint_as_float(r[j]) + b4[cb + j], __uint_as_float(r[j + 1]) + b4[cb + j + 1]);
                s += __uint_as_float(pk[e] << 16) * w5[cb + j] + __uint_as_float(pk[e] & 0xFFFF0000u) * w5[cb + j + 1];
                if (TRAIN) bits |= pos_bits(pk[e]) << j;
            }
            if (TRAIN)
                *reinterpret_cast<uint4 *>(ws_blk + act_row(row) + ((cb >> 3) + q) * 128) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        if (TRAIN) ws_mask[row * 4 + (cb >> 5)] = bits;
    }
    return s;
}

// Row `row` of the pooling matrix S, k in [c0, c0 + 64), into 32 TMEM columns of bfloat16
// pairs: S[row][k] = 1 when rows row and k belong to the same race (r0 <= k < r1; a zero row
// for padding), so that S . h3 sums h3 over the race of every row.
__device__ __forceinline__ void tc_store_pool_row(uint32_t taddr_s, int r0, int r1, int c0)
{
    const uint32_t n = uint32_t(r1 - r0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t t = uint32_t(c0 + 32 * h + 2 * j - r0);  // k - r0, wrapping below r0
            v[j] = (t < n ? 0x3F80u : 0u) | (t + 1u < n ? 0x3F800000u : 0u);
        }
        tmem_st16<0>(taddr_s + c0 / 2 + 16 * h, v);
    }
}

// pooled sums (TMEM accumulator columns [c0, c0 + 64)) -> g = bfloat16(sum x inv_n) -> 32
// TMEM columns of bfloat16 pairs, the A operand of the head's second product (and the
// workspace block when training)
template <bool TRAIN>
__device__ __forceinline__ void tc_epilogue_pool(uint32_t taddr_d, uint32_t taddr_g, float inv_n, int row,
                                                 unsigned char *ws_blk, int c0)
{
#pragma unroll
    for (int cb = c0; cb < c0 + 64; cb += 32) {
        uint32_t r[32];
        tmem_ld16<0>(r, taddr_d + cb);
        tmem_ld16<16>(r, taddr_d + cb + 16);
        tmem_wait_ld();
        uint32_t g[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            g[j] = pack_bf16x2(__uint_as_float(r[2 * j]) * inv_n, __uint_as_float(r[2 * j + 1]) * inv_n);
        tmem_st16<0>(taddr_g + cb / 2, g);
        if (TRAIN) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<uint4 *>(ws_blk + act_row(row) + ((cb >> 3) + q) * 128) =
                    make_uint4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
        }
    }
}

struct __align__(128) TcPipe {
    unsigned char xb[2][TILE * KIN * 2];  // features of this and the next tile, canonical K-major (K = 16)
    TileMeta mt[2];                       // their race layout
    unsigned char act[TILE * H * 2];      // h1, h2, h3, then g (canonical, K = 128)
    unsigned long long mbar_in[2];        // bulk copies of xb[i], mt[i]
    float logit_part[2][TILE];            // the two column halves of w5 . u
};

struct TcSmem {
    unsigned char w[WC_ELEMS * 2];  // W1, W2, W3, W4 (canonical image)
    TcPipe pipe[2];
    float bias[4][H];               // b1, b2, b3, b4
    float w5[H];
    float b5;
    int abort[2];
    uint32_t tmem_base;
    unsigned long long mbar_w, mbar[2];
};
static_assert(sizeof(TcSmem) <= 227 * 1024, "forward shared memory");
static_assert(sizeof(TileMeta) % 16 == 0, "tile layout records are moved by bulk copies");

// wait for this pipeline's product; on a timeout flag the pipeline and the launch
__device__ __forceinline__ bool group_wait(TcSmem &sm, int wg, uint32_t &phase, const SgArgs &a)
{
    // warp-uniform, since the epilogue's tensor-memory loads are warp-collective
    const bool done = __all_sync(0xffffffffu, mbar_wait(&sm.mbar[wg], phase, a.wait_ns));
    phase ^= 1u;
    if (!done) {
        *reinterpret_cast<volatile int *>(&sm.abort[wg]) = 1;
        atomicOr(a.status, 1);
    }
    tc_after_sync();
    return done;
}

// bulk copies of tile ti's features and race layout into buffer i of the pipeline
__device__ __forceinline__ void load_tile_inputs(TcPipe &P, int i, int ti, const SgArgs &a)
{
    mbar_expect_tx(&P.mbar_in[i], uint32_t(TILE * KIN * 2 + sizeof(TileMeta)));
    bulk_g2s(P.xb[i], a.xbuf + size_t(ti) * (TILE * KIN * 2), TILE * KIN * 2, &P.mbar_in[i]);
    bulk_g2s(&P.mt[i], a.meta + ti, uint32_t(sizeof(TileMeta)), &P.mbar_in[i]);
}

// Tile features and race layout (one 128-thread block per tile): x in the canonical operand
// layout (also the training pass's x), the tile's race layout record.
// Programmatic dependent launch (the step's kernels go out with
// cudaLaunchAttributeProgrammaticStreamSerialization): let the next kernel on the stream be
// scheduled as soon as every block of this one has started, then wait until the kernels before
// this one have completed and their writes are visible.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__global__ void __launch_bounds__(TILE) sg_prep(SgArgs a)
{
    pdl_enter();
    __shared__ RowMap m;
    __shared__ FeatScratch fs;
    const int tid = threadIdx.x, ti = blockIdx.x;
    const SgTile t = a.tiles[ti];
    build_rowmap(m, a, t, tid, BlockSync{});
    float f[KIN];
    tile_features(f, fs, a, m, tid, BlockSync{});
    if (a.raw_only) {
#pragma unroll
        for (int k = RAW; k < KIN; ++k) f[k] = 0.0f;
    }
    const uint4 lo = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                                pack_bf16x2(f[6], f[7]));
    const uint4 hi = make_uint4(pack_bf16x2(f[8], f[9]), pack_bf16x2(f[10], f[11]), pack_bf16x2(f[12], f[13]),
                                pack_bf16x2(f[14], f[15]));
    unsigned char *xt = a.xbuf + size_t(ti) * (TILE * KIN * 2);
    *reinterpret_cast<uint4 *>(xt + canon_off(tid, 0, KIN)) = lo;
    *reinterpret_cast<uint4 *>(xt + canon_off(tid, 8, KIN)) = hi;
    TileMeta &mt = a.meta[ti];
    if (tid == 0) {
        mt.ns = t.ns;
        mt.nrows = t.nrows;
    }
    if (tid <= t.ns) mt.state_row0[tid] = m.state_row0[tid];
    if (tid < t.ns) mt.state_race[tid] = m.state_race[tid];
    mt.row_state[tid] = int8_t(m.row_race[tid] >= 0 ? m.row_state[tid] : -1);
}

template <bool TRAIN>
__global__ void __launch_bounds__(TC_THREADS, 1) sg_forward_tc(SgArgs a, int n_tiles)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = tid / TC_PIPE, pt = tid % TC_PIPE;  // pipeline, thread within it
    const int ch = (pt >> 7) & 1;                     // column half of this thread
    TcPipe &P = sm.pipe[p];
    const GroupSync sync{1 + p, TC_PIPE};
    volatile int *abort_flag = &sm.abort[p];
    const int first = p * gridDim.x + blockIdx.x, stride = 2 * gridDim.x;

    if (pt == 0) {
        if (p == 0) {
            mbar_init(&sm.mbar_w, 1);
            sm.abort[0] = sm.abort[1] = 0;
        }
        mbar_init(&sm.mbar[p], 1);
        mbar_init(&P.mbar_in[0], 1);
        mbar_init(&P.mbar_in[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(4 * H)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 4 * H; i += TC_THREADS) {
        const int l = i / H, c = i - l * H;
        sm.bias[l][c] = a.wf[(l == 0 ? OFF_B1 : l == 1 ? OFF_B2 : l == 2 ? OFF_B3 : OFF_B4) + c];
    }
    if (tid < H) sm.w5[tid] = a.wf[OFF_W5 + tid];
    if (tid == 0) sm.b5 = a.wf[OFF_B5];
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
        mbar_expect_tx(&sm.mbar_w, WC_ELEMS * 2);
        bulk_g2s(sm.w + WC_W1 * 2, a.wc + WC_W1, (WC_W2 - WC_W1) * 2, &sm.mbar_w);
        bulk_g2s(sm.w + WC_W2 * 2, a.wc + WC_W2, (WC_W3 - WC_W2) * 2, &sm.mbar_w);
        bulk_g2s(sm.w + WC_W3 * 2, a.wc + WC_W3, (WC_W4 - WC_W3) * 2, &sm.mbar_w);
        bulk_g2s(sm.w + WC_W4 * 2, a.wc + WC_W4, (WC_ELEMS - WC_W4) * 2, &sm.mbar_w);
    }
    if (pt == 0 && first < n_tiles) load_tile_inputs(P, 0, first, a);

    // this pipeline's 256 TMEM columns: accumulator D [0, 128), pooling matrix S [128, 192),
    // context g [192, 256); this warp reads and writes lanes 32 (warp % 4) .. 32 (warp % 4) + 31
    const uint32_t tmem = sm.tmem_base + uint32_t(p * 2 * H);
    const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;
    const uint32_t td = tmem + lane_off, ts = tmem + H + lane_off, tg = tmem + H + H / 2 + lane_off;
    const uint32_t sact = smem_addr(P.act), sw = smem_addr(sm.w);
    const int row = (warp & 3) * 32 + lane;  // tile row of this thread = its TMEM lane
    const int c0 = ch * (H / 2);             // first accumulator column of this thread
    uint32_t phase = 0;
    bool weights_ready = false;
    int pending = first < n_tiles ? 0 : -1;  // input buffer with a copy in flight (issuing thread)
    uint32_t pending_parity = 0;

    int k = 0;
    for (int ti = first; ti < n_tiles; ti += stride, ++k) {
        const int ib = k & 1;
        const uint32_t in_parity = uint32_t(k >> 1) & 1u;
        const bool in_ok = __all_sync(0xffffffffu, mbar_wait(&P.mbar_in[ib], in_parity, a.wait_ns));
        if (!in_ok) {
            *abort_flag = 1;
            atomicOr(a.status, 1);
        }
        unsigned char *ws = TRAIN ? a.ws + size_t(ti) * WS_TILE : nullptr;
        uint32_t *wsm = ws ? reinterpret_cast<uint32_t *>(ws + WS_M) : nullptr;  // masks of h1, h2, h3, u
        const TileMeta &mt = P.mt[ib];

        // layer 1: h1 = relu(W1 x + b1); the next tile's inputs are fetched meanwhile
        if (pt == 0) {
            pending = -1;
            const bool have_w = weights_ready || mbar_wait(&sm.mbar_w, 0, a.wait_ns);
            tc_after_sync();
            if (have_w && in_ok) {
                if (ti + stride < n_tiles) {
                    load_tile_inputs(P, ib ^ 1, ti + stride, a);
                    pending = ib ^ 1;
                    pending_parity = uint32_t((k + 1) >> 1) & 1u;
                }
                tc_mma(tmem, smem_desc(smem_addr(P.xb[ib]), 128, 2 * 128), smem_desc(sw + WC_W1 * 2, 128, 2 * 128), 0u);
                tc_commit(&sm.mbar[p]);
            } else {
                *abort_flag = 1;
                atomicOr(a.status, 1);
                mbar_arrive(&sm.mbar[p]);  // release the pipeline's waiters
            }
        }
        weights_ready = true;
        // meanwhile: this row's part of the pooling matrix and its race's 1 / n
        float inv_n = 0.0f;
        {
            const int st = in_ok ? mt.row_state[row] : -1;
            int r0 = 0, r1 = 0;
            if (st >= 0) {
                r0 = mt.state_row0[st];
                r1 = mt.state_row0[st + 1];
                inv_n = 1.0f / float(r1 - r0);
            }
            tc_store_pool_row(ts, r0, r1, c0);
            tmem_wait_st();
        }
        if (group_wait(sm, p, phase, a))
            tc_epilogue_relu<TRAIN>(td, sm.bias[0], P.act, row, ws ? ws + WS_H1 : nullptr, wsm, c0);
        fence_async_smem();
        tc_before_sync();
        sync();
        if (*abort_flag) break;

        // layers 2 and 3: h = relu(W h_prev + b), in place
        for (int l = 1; l <= 2; ++l) {
            if (pt == 0) {
                tc_after_sync();
                const uint32_t wl = sw + uint32_t(l == 1 ? WC_W2 : WC_W3) * 2;
#pragma unroll
                for (int ks = 0; ks < H / 16; ++ks)
                    tc_mma(tmem, smem_desc(sact + ks * 256, 128, 16 * 128), smem_desc(wl + ks * 256, 128, 16 * 128),
                           ks > 0 ? 1u : 0u);
                tc_commit(&sm.mbar[p]);
            }
            if (group_wait(sm, p, phase, a))
                tc_epilogue_relu<TRAIN>(td, sm.bias[l], P.act, row, ws ? ws + WS_H1 + l * WS_BLOCK : nullptr,
                                 wsm ? wsm + l * (WS_MASK / 4) : nullptr, c0);
            fence_async_smem();
            tc_before_sync();
            sync();
            if (*abort_flag) break;
        }
        if (*abort_flag) break;

        // pooled sums S . h3: A = S from tensor memory, B = h3^T, i.e. the activation tile read
        // as an MN-major operand (core matrices 16 B apart along N, 2048 B apart along K)
        if (pt == 0) {
            tc_after_sync();
#pragma unroll
            for (int ks = 0; ks < TILE / 16; ++ks)
                tc_mma_ta(tmem, tmem + H + ks * 8, smem_desc(sact + ks * 4096, 2048, 128), kIdescBmn, ks > 0 ? 1u : 0u);
            tc_commit(&sm.mbar[p]);
        }
        if (group_wait(sm, p, phase, a)) tc_epilogue_pool<TRAIN>(td, tg, inv_n, row, ws ? ws + WS_G : nullptr, c0);
        tmem_wait_st();
        tc_before_sync();
        sync();
        if (*abort_flag) break;

        // head: h3 . W4[:, 0:128]^T + g . W4[:, 128:256]^T; u = relu(. + b4), logit = w5 . u + b5
        if (pt == 0) {
            tc_after_sync();
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks)
                tc_mma(tmem, smem_desc(sact + ks * 256, 128, 16 * 128), smem_desc(sw + WC_W4 * 2 + ks * 256, 128, 32 * 128),
                       ks > 0 ? 1u : 0u);
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks)
                tc_mma_ta(tmem, tmem + H + H / 2 + ks * 8, smem_desc(sw + WC_W4 * 2 + (H / 16 + ks) * 256, 128, 32 * 128),
                          kIdesc, 1u);
            tc_commit(&sm.mbar[p]);
        }
        if (group_wait(sm, p, phase, a))
            P.logit_part[ch][row] =
                tc_epilogue_head<TRAIN>(td, sm.bias[3], sm.w5, row, ws ? ws + WS_U : nullptr, wsm ? wsm + 3 * (WS_MASK / 4) : nullptr,
                                 c0);
        fence_async_smem();
        tc_before_sync();
        sync();
        if (*abort_flag) break;
        if (ch == 0) a.logits[size_t(ti) * TILE + row] = P.logit_part[0][row] + P.logit_part[1][row] + sm.b5;
    }
    // a copy still in flight after an abort: wait for it before the block's memory goes
    if (pt == 0 && pending >= 0) mbar_wait(&P.mbar_in[pending], pending_parity, a.wait_ns);
    if (tid == 0 && !weights_ready) mbar_wait(&sm.mbar_w, 0, a.wait_ns);
    // every product this block issued has been waited for (or its wait gave up)
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base), "r"(4 * H) : "memory");
    }
}

// inference softmax: one warp per tile, one lane per race (its rows in row order); measured
// faster than one thread per row when there are many tiles and no loss to reduce
__global__ void sg_softmax_infer(SgArgs a, int n_tiles)
{
    pdl_enter();
    const int ti = int((blockIdx.x * size_t(blockDim.x) + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (ti >= n_tiles) return;
    const TileMeta &mt = a.meta[ti];
    const float *lg = a.logits + size_t(ti) * TILE;
    for (int st = lane; st < mt.ns; st += 32) {
        const int r0 = mt.state_row0[st], r1 = mt.state_row0[st + 1];
        const int base = a.b.race_off[mt.state_race[st]];
        float mx = -INFINITY;
        for (int q = r0; q < r1; ++q) mx = fmaxf(mx, lg[q]);
        float sum = 0.0f;
        for (int q = r0; q < r1; ++q) sum += expf(lg[q] - mx);
        const float lsum = logf(sum);
        for (int q = r0; q < r1; ++q) a.probs[base + (q - r0)] = expf(lg[q] - mx - lsum);
    }
}

// softmax over each race's logits; training: the loss and d loss / d logit per tile row (zero
// on padding rows).  One block per tile, one thread per row: the tile's logits and race layout
// in shared memory, each row's thread takes its race's maximum and sum over the race's rows in
// row order, then writes its own probability (and, in training, d loss / d logit).
__global__ void __launch_bounds__(TILE) sg_softmax(SgArgs a, int n_tiles)
{
    pdl_enter();
    __shared__ float lg[TILE];
    __shared__ int32_t row0[MAX_STATES + 1];
    __shared__ float red[TILE / 32];
    const int ti = blockIdx.x, q = threadIdx.x;
    if (ti >= n_tiles) return;
    const TileMeta &mt = a.meta[ti];
    const int ns = mt.ns;
    lg[q] = a.logits[size_t(ti) * TILE + q];
    if (q <= ns) row0[q] = mt.state_row0[q];
    const int st = mt.row_state[q];
    __syncthreads();
    float lossv = 0.0f, dl = 0.0f;
    if (st >= 0) {
        const int r0 = row0[st], r1 = row0[st + 1];
        const int base = a.b.race_off[mt.state_race[st]];
        float mx = -INFINITY;
        for (int j = r0; j < r1; ++j) mx = fmaxf(mx, lg[j]);
        float sum = 0.0f;
        for (int j = r0; j < r1; ++j) sum += expf(lg[j] - mx);
        const float lq = lg[q] - mx - logf(sum);  // log q
        const float qv = expf(lq);
        if (a.probs) a.probs[base + (q - r0)] = qv;
        if (a.train) {
            float tsum = 0.0f;
            for (int j = r0; j < r1; ++j) tsum += a.target[base + (j - r0)];
            const float tv = a.target[base + (q - r0)];
            dl = (qv * tsum - tv) * a.inv_races;
            lossv = -tv * lq;
        }
    }
    if (a.train) {
        a.ws_dlogit[size_t(ti) * TILE + q] = dl;  // 0 on padding rows
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lossv += __shfl_xor_sync(0xffffffffu, lossv, o);
        if ((q & 31) == 0) red[q >> 5] = lossv;
        __syncthreads();
        if (q == 0 && a.loss_acc) atomicAdd(a.loss_acc, (red[0] + red[1] + red[2] + red[3]) * a.inv_races);
    }
}

// ------------------------------------------------------------------ backward (tcgen05)
//
// Two persistent kernels and a reduction.  The forward pass of a training step leaves, per tile,
// h1, h2, h3, g and u in the canonical activation layout, the ReLU masks of h1, h2, h3 and u as
// bits, and d loss / d logit per row.
//   sg_backward_chain   one 256-thread block per SM, W2, W3, W4 resident in shared memory,
//                       the tile's masks and d logit by bulk copy (double-buffered):
//                         du  = dlogit w5 [u > 0]                         (CUDA cores)
//                         dz  = du . W4          (tcgen05, N = 256: W4 read as an MN-major B)
//                         pooled context gradient S . dz_g (S, the race indicator, in TMEM;
//                             dz_g rounded to bfloat16 in shared memory as an MN-major B)
//                         da3 = (dz_h + pooled / n) [h3 > 0]
//                         da2 = (da3 . W3) [h2 > 0],  da1 = (da2 . W2) [h1 > 0]
//                       du, da3, da2, da1 go to the workspace in bfloat16.
//   sg_backward_wgrad   split-K over tiles: block group 0 accumulates dW4 = du^T [h3 ; g], the
//                       b4 gradient (du^T . 1) and the w5 gradient (u^T . dlogit, dlogit split
//                       into two bfloat16 parts) in tensor memory over its tiles; group 1
//                       dW3 = da3^T h2, dW2 = da2^T h1, dW1 = da1^T x and the b3, b2, b1
//                       gradients.  The transposed operands are the workspace blocks read as
//                       MN-major operands.  Each block writes its partial sums once.
//   sg_reduce_grad      the float32 gradient = sum of the blocks' partials in block order.
// The b5 gradient (sum of d logit) is added by the chain kernel.

// instruction descriptor with M = 128, N = n, bfloat16 in, float32 out; a_mn / b_mn: MN-major
__host__ __device__ constexpr uint32_t idesc_of(int n, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(a_mn) << 15) | (uint32_t(b_mn) << 16) |
           (uint32_t(n >> 3) << 17) | (uint32_t(TILE >> 4) << 24);
}

// D (+)= A . B^T with both operands in shared memory and an explicit instruction descriptor
__device__ __forceinline__ void tc_mma_d(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

struct __align__(16) BcIn {
    uint32_t mask[4][TILE][4];  // masks of h1, h2, h3, u
    float dlogit[TILE];
    TileMeta mt;
};
static_assert(sizeof(BcIn) % 16 == 0 && sizeof(BcIn) == 4 * WS_MASK + TILE * 4 + sizeof(TileMeta), "chain inputs");

struct BcSmem {
    unsigned char w4[H * 2 * H * 2];  // canonical W4, W3, W2 (rows = outputs)
    unsigned char w3[H * H * 2];
    unsigned char w2[H * H * 2];
    unsigned char buf[TILE * H * 2];  // du, then dz_g, da3, da2 (canonical activation layout)
    BcIn in[2];
    float w5[H];
    int abort;
    uint32_t tmem_base;
    unsigned long long mbar_w, mbar, mbar_in[2];
};
static_assert(sizeof(BcSmem) <= 227 * 1024, "chain shared memory");

__device__ __forceinline__ void load_chain_inputs(BcSmem &sm, int i, int ti, const SgArgs &a)
{
    mbar_expect_tx(&sm.mbar_in[i], uint32_t(sizeof(BcIn)));
    bulk_g2s(sm.in[i].mask, a.ws + size_t(ti) * WS_TILE + WS_M, uint32_t(4 * WS_MASK), &sm.mbar_in[i]);
    bulk_g2s(sm.in[i].dlogit, a.ws_dlogit + size_t(ti) * TILE, TILE * 4, &sm.mbar_in[i]);
    bulk_g2s(&sm.in[i].mt, a.meta + ti, uint32_t(sizeof(TileMeta)), &sm.mbar_in[i]);
}

// wait for the block's product; a timeout flags the block and the launch
__device__ __forceinline__ bool block_wait(unsigned long long *bar, uint32_t &phase, int *abort, const SgArgs &a)
{
    const bool done = __all_sync(0xffffffffu, mbar_wait(bar, phase, a.wait_ns));
    phase ^= 1u;
    if (!done) {
        *reinterpret_cast<volatile int *>(abort) = 1;
        atomicOr(a.status, 1);
    }
    tc_after_sync();
    return done;
}

// 32 float32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t (&r)[32], uint32_t taddr)
{
    tmem_ld16<0>(r, taddr);
    tmem_ld16<16>(r, taddr + 16);
    tmem_wait_ld();
}

__global__ void __launch_bounds__(256, 1) sg_backward_chain(SgArgs a, int n_tiles)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BcSmem &sm = *reinterpret_cast<BcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = (warp & 3) * 32 + lane;  // TMEM lane = tile row
    const int c0 = (warp >> 2) * 64;         // this thread's 64 columns
    volatile int *abort_flag = &sm.abort;
    if (tid == 0) {
        mbar_init(&sm.mbar_w, 1);
        mbar_init(&sm.mbar, 1);
        mbar_init(&sm.mbar_in[0], 1);
        mbar_init(&sm.mbar_in[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(4 * H)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < H) sm.w5[tid] = a.wf[OFF_W5 + tid];
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const int first = blockIdx.x, stride = gridDim.x;
    if (tid == 0) {
        mbar_expect_tx(&sm.mbar_w, uint32_t((WC_ELEMS - WC_W2) * 2));
        bulk_g2s(sm.w2, a.wc + WC_W2, (WC_W3 - WC_W2) * 2, &sm.mbar_w);
        bulk_g2s(sm.w3, a.wc + WC_W3, (WC_W4 - WC_W3) * 2, &sm.mbar_w);
        bulk_g2s(sm.w4, a.wc + WC_W4, (WC_ELEMS - WC_W4) * 2, &sm.mbar_w);
        if (first < n_tiles) load_chain_inputs(sm, 0, first, a);
    }
    // tensor memory: dz [0, 256) (dz_h, dz_g), pooled [256, 384), S [384, 448)
    const uint32_t tmem = sm.tmem_base;
    const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;
    const uint32_t tdz = tmem + lane_off, tpool = tmem + 256 + lane_off, ts = tmem + 384 + lane_off;
    const uint32_t sbuf = smem_addr(sm.buf);
    unsigned char *brow = sm.buf + act_row(row);
    uint32_t phase = 0;
    bool weights_ready = false;
    int pending = first < n_tiles ? 0 : -1;
    uint32_t pending_parity = 0;

    int k = 0;
    for (int ti = first; ti < n_tiles; ti += stride, ++k) {
        const int ib = k & 1;
        const bool in_ok = __all_sync(0xffffffffu, mbar_wait(&sm.mbar_in[ib], uint32_t(k >> 1) & 1u, a.wait_ns));
        if (!in_ok) {
            *abort_flag = 1;
            atomicOr(a.status, 1);
        }
        const BcIn &in = sm.in[ib];
        unsigned char *ws = a.ws + size_t(ti) * WS_TILE;
        if (tid == 0) {
            pending = -1;
            if (in_ok && ti + stride < n_tiles) {
                load_chain_inputs(sm, ib ^ 1, ti + stride, a);
                pending = ib ^ 1;
                pending_parity = uint32_t((k + 1) >> 1) & 1u;
            }
            if (!weights_ready && !mbar_wait(&sm.mbar_w, 0, a.wait_ns)) {
                *abort_flag = 1;
                atomicOr(a.status, 1);
            }
        }
        weights_ready = true;
        // this row's part of the race indicator S (zero row for padding) and its race's 1 / n
        float inv_n = 0.0f;
        {
            const int st = in_ok ? in.mt.row_state[row] : -1;
            int r0 = 0, r1 = 0;
            if (st >= 0) {
                r0 = in.mt.state_row0[st];
                r1 = in.mt.state_row0[st + 1];
                inv_n = 1.0f / float(r1 - r0);
            }
            tc_store_pool_row(ts, r0, r1, c0);
            tmem_wait_st();
        }
        // du = dlogit w5 [u > 0]
        {
            const float dl = in.dlogit[row];
#pragma unroll
            for (int cb = c0; cb < c0 + 64; cb += 32) {
                const uint32_t mu4 = in.mask[3][row][cb >> 5];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t pk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = q * 8 + 2 * e;
                        const float lo = (mu4 >> j) & 1u ? __fmul_rn(dl, sm.w5[cb + j]) : 0.0f;
                        const float hi = (mu4 >> (j + 1)) & 1u ? __fmul_rn(dl, sm.w5[cb + j + 1]) : 0.0f;
                        pk[e] = pack_bf16x2(lo, hi);
                    }
                    const uint4 v = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4 *>(brow + ((cb >> 3) + q) * 128) = v;
                    *reinterpret_cast<uint4 *>(ws + WS_DU + act_row(row) + ((cb >> 3) + q) * 128) = v;
                }
            }
        }
        if (tid == 0 && in_ok) {
            // this tile's term of the b5 gradient; the reduction adds the tiles in order
            float sdl = 0.0f;
            for (int q = 0; q < TILE; ++q) sdl += in.dlogit[q];
            a.b5_part[ti] = sdl;
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (*abort_flag) break;

        // dz = du . W4 (B = W4 read MN-major: rows = outputs are the reduction, inputs the N side)
        if (tid == 0) {
            tc_after_sync();
            const uint32_t w4 = smem_addr(sm.w4);
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks)
                tc_mma_d(tmem, smem_desc(sbuf + ks * 256, 128, 16 * 128), smem_desc(w4 + ks * 8192, 4096, 128),
                         idesc_of(2 * H, 0, 1), ks > 0 ? 1u : 0u);
            tc_commit(&sm.mbar);
        }
        if (block_wait(&sm.mbar, phase, &sm.abort, a)) {
            // dz_g -> bfloat16 over du (the product has read it)
#pragma unroll
            for (int cb = c0; cb < c0 + 64; cb += 32) {
                uint32_t r[32];
                tmem_ld32(r, tdz + H + cb);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4 *>(brow + ((cb >> 3) + q) * 128) =
                        make_uint4(pack_bf16x2(__uint_as_float(r[8 * q]), __uint_as_float(r[8 * q + 1])),
                                   pack_bf16x2(__uint_as_float(r[8 * q + 2]), __uint_as_float(r[8 * q + 3])),
                                   pack_bf16x2(__uint_as_float(r[8 * q + 4]), __uint_as_float(r[8 * q + 5])),
                                   pack_bf16x2(__uint_as_float(r[8 * q + 6]), __uint_as_float(r[8 * q + 7])));
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (*abort_flag) break;

        // per-race sums of dz_g: S . dz_g (A = S in tensor memory, B = dz_g^T read MN-major)
        if (tid == 0) {
            tc_after_sync();
#pragma unroll
            for (int ks = 0; ks < TILE / 16; ++ks)
                tc_mma_ta(tmem + 256, tmem + 384 + ks * 8, smem_desc(sbuf + ks * 4096, 2048, 128), kIdescBmn,
                          ks > 0 ? 1u : 0u);
            tc_commit(&sm.mbar);
        }
        if (block_wait(&sm.mbar, phase, &sm.abort, a)) {
            // da3 = (dz_h + pooled / n) [h3 > 0]
#pragma unroll
            for (int cb = c0; cb < c0 + 64; cb += 32) {
                uint32_t rz[32], rp[32];
                tmem_ld32(rz, tdz + cb);
                tmem_ld32(rp, tpool + cb);
                const uint32_t m3 = in.mask[2][row][cb >> 5];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t pk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = q * 8 + 2 * e;
                        const float lo = (m3 >> j) & 1u ? __fmaf_rn(__uint_as_float(rp[j]), inv_n, __uint_as_float(rz[j])) : 0.0f;
                        const float hi = (m3 >> (j + 1)) & 1u
                                             ? __fmaf_rn(__uint_as_float(rp[j + 1]), inv_n, __uint_as_float(rz[j + 1]))
                                             : 0.0f;
                        pk[e] = pack_bf16x2(lo, hi);
                    }
                    const uint4 v = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4 *>(brow + ((cb >> 3) + q) * 128) = v;
                    *reinterpret_cast<uint4 *>(ws + WS_DA3 + act_row(row) + ((cb >> 3) + q) * 128) = v;
                }
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (*abort_flag) break;

        // da2 = (da3 . W3) [h2 > 0], then da1 = (da2 . W2) [h1 > 0]
        for (int l = 0; l < 2; ++l) {
            if (tid == 0) {
                tc_after_sync();
                const uint32_t wl = smem_addr(l == 0 ? sm.w3 : sm.w2);
#pragma unroll
                for (int ks = 0; ks < H / 16; ++ks)
                    tc_mma_d(tmem, smem_desc(sbuf + ks * 256, 128, 16 * 128), smem_desc(wl + ks * 4096, 2048, 128),
                             idesc_of(H, 0, 1), ks > 0 ? 1u : 0u);
                tc_commit(&sm.mbar);
            }
            if (block_wait(&sm.mbar, phase, &sm.abort, a)) {
#pragma unroll
                for (int cb = c0; cb < c0 + 64; cb += 32) {
                    uint32_t r[32];
                    tmem_ld32(r, tdz + cb);
                    const uint32_t mk = in.mask[1 - l][row][cb >> 5];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = q * 8 + 2 * e;
                            pk[e] = pack_bf16x2((mk >> j) & 1u ? __uint_as_float(r[j]) : 0.0f,
                                                (mk >> (j + 1)) & 1u ? __uint_as_float(r[j + 1]) : 0.0f);
                        }
                        const uint4 v = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        if (l == 0) *reinterpret_cast<uint4 *>(brow + ((cb >> 3) + q) * 128) = v;
                        *reinterpret_cast<uint4 *>(ws + (l == 0 ? WS_DA2 : WS_DA1) + act_row(row) + ((cb >> 3) + q) * 128) = v;
                    }
                }
            }
            fence_async_smem();
            tc_before_sync();
            __syncthreads();
            if (*abort_flag) break;
        }
        if (*abort_flag) break;
    }
    if (tid == 0 && pending >= 0) mbar_wait(&sm.mbar_in[pending], pending_parity, a.wait_ns);
    if (tid == 0 && !weights_ready) mbar_wait(&sm.mbar_w, 0, a.wait_ns);
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base), "r"(4 * H) : "memory");
    }
}

// The weight-gradient kernel streams each tile through shared memory in quarters (32 rows of the
// reduction) through WG_SLOTS slots: while the tensor cores work on quarter u (and may still be on
// u - 1), the copies of quarters u + 1 .. u + WG_AHEAD are on their way.
constexpr int WG_SLOTS = 4;
constexpr int WG_AHEAD = WG_SLOTS - 2;                    // quarters fetched ahead of the one in use
constexpr int WG_ROWS = TILE / 4;                         // rows of one quarter
constexpr uint32_t WS_QTR = uint32_t(WS_BLOCK / 4);       // 32 rows of a canonical block

struct BwSmem {
    // WG_SLOTS slots, each one quarter of a tile: group 0 du, h3, g, u; group 1 da3, h2, da2, h1,
    // da1; plus x (group 1) and d logit (group 0) of that quarter
    unsigned char blk[WG_SLOTS][5][WS_QTR];
    unsigned char x[WG_SLOTS][WG_ROWS * KIN * 2];  // 32 rows of x (canonical, K = 16)
    float dlogit[WG_SLOTS][WG_ROWS];
    unsigned char ones[16 * TILE * 2];   // B operand [16][128 rows]: row 0 ones, the rest zeros
    unsigned char dls[16 * TILE * 2];    // group 0: B operand, rows 0 and 1 the two bfloat16 parts of dlogit
    int abort;
    uint32_t tmem_base;
    unsigned long long mbar_mma[WG_SLOTS], mbar_in[WG_SLOTS];
};
static_assert(sizeof(BwSmem) <= 227 * 1024, "weight-gradient shared memory");

// byte offset of element (n, k) of a canonical K-major [16][128] operand
__device__ __forceinline__ uint32_t nk_off(int n, int k) { return canon_off(n, k, TILE); }

// bulk copies of quarter `part` (rows 32 part ..) of tile ti into slot `slot`
__device__ __forceinline__ void load_wgrad_quarter(BwSmem &sm, int slot, int group, int ti, int part, const SgArgs &a)
{
    const unsigned char *ws = a.ws + size_t(ti) * WS_TILE + size_t(part) * WS_QTR;
    unsigned long long *bar = &sm.mbar_in[slot];
    if (group == 0) {
        mbar_expect_tx(bar, 4 * WS_QTR + WG_ROWS * 4);
        bulk_g2s(sm.blk[slot][0], ws + WS_DU, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][1], ws + WS_H1 + 2 * WS_BLOCK, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][2], ws + WS_G, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][3], ws + WS_U, WS_QTR, bar);
        bulk_g2s(sm.dlogit[slot], a.ws_dlogit + size_t(ti) * TILE + part * WG_ROWS, WG_ROWS * 4, bar);
    } else {
        mbar_expect_tx(bar, 5 * WS_QTR + WG_ROWS * KIN * 2);
        bulk_g2s(sm.blk[slot][0], ws + WS_DA3, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][1], ws + WS_H1 + WS_BLOCK, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][2], ws + WS_DA2, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][3], ws + WS_H1, WS_QTR, bar);
        bulk_g2s(sm.blk[slot][4], ws + WS_DA1, WS_QTR, bar);
        bulk_g2s(sm.x[slot], a.xbuf + size_t(ti) * (TILE * KIN * 2) + part * (WG_ROWS * KIN * 2), WG_ROWS * KIN * 2, bar);
    }
}

__global__ void __launch_bounds__(128, 1) sg_backward_wgrad(SgArgs a, int n_tiles)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BwSmem &sm = *reinterpret_cast<BwSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int group = blockIdx.x / a.wgroups, cta = blockIdx.x % a.wgroups;
    volatile int *abort_flag = &sm.abort;
    if (tid == 0) {
        for (int i = 0; i < WG_SLOTS; ++i) {
            mbar_init(&sm.mbar_mma[i], 1);
            mbar_init(&sm.mbar_in[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(4 * H)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // constant operands: ones in row 0, zeros elsewhere (rows 0 and 1 of dls are rewritten per quarter)
    for (int i = tid; i < 16 * TILE; i += 128) {
        const int n = i / TILE, kk = i - n * TILE;
        *reinterpret_cast<bf16 *>(sm.ones + nk_off(n, kk)) = __float2bfloat16_rn(n == 0 ? 1.0f : 0.0f);
        *reinterpret_cast<bf16 *>(sm.dls + nk_off(n, kk)) = __float2bfloat16_rn(0.0f);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = sm.tmem_base;
    const uint32_t sones = smem_addr(sm.ones), sdls = smem_addr(sm.dls);
    // this block's quarters: u = 0 .. n_q-1 is quarter (u & 3) of its (u >> 2)-th tile
    const int my_tiles = cta < n_tiles ? (n_tiles - 1 - cta) / a.wgroups + 1 : 0;
    const int n_q = 4 * my_tiles;
    // per slot, one bit each (registers, not an indexed array): the phase of its product and copy
    // barriers, and (issuing thread) a copy not yet waited for with the phase it completes
    uint32_t mma_bits = 0u, in_bits = 0u, pend_bits = 0u, pend_par = 0u;
    auto wait_slot = [&](unsigned long long *bar, uint32_t &bits, int i) {
        uint32_t ph = (bits >> i) & 1u;
        const bool done = block_wait(bar, ph, &sm.abort, a);
        bits ^= 1u << i;
        return done;
    };
    auto note_copy = [&](int i) {
        pend_bits |= 1u << i;
        pend_par = (pend_par & ~(1u << i)) | (in_bits & (1u << i));
    };
    if (tid == 0) {
        for (int u = 0; u < WG_AHEAD && u < n_q; ++u) {
            load_wgrad_quarter(sm, u, group, cta + (u >> 2) * a.wgroups, u & 3, a);
            note_copy(u);
        }
    }
    int done_q = 0;
    for (int u = 0; u < n_q; ++u) {
        const int slot = u % WG_SLOTS, part = u & 3;
        // fetch quarter u + WG_AHEAD into the slot of quarter u + WG_AHEAD - WG_SLOTS, once that
        // quarter's product has finished (the product of u - 1 may still be running)
        const int nxt = u + WG_AHEAD, nslot = nxt % WG_SLOTS;
        if (nxt < n_q) {
            if (nxt >= WG_SLOTS && !wait_slot(&sm.mbar_mma[nslot], mma_bits, nslot)) break;
            if (tid == 0) {
                load_wgrad_quarter(sm, nslot, group, cta + (nxt >> 2) * a.wgroups, nxt & 3, a);
                note_copy(nslot);
            }
        }
        if (!wait_slot(&sm.mbar_in[slot], in_bits, slot)) break;
        pend_bits &= ~(1u << slot);
        if (group == 0 && tid < WG_ROWS) {
            // d logit of these 32 rows as two bfloat16 parts (hi + lo) in rows 0 and 1 of dls
            const float dl = sm.dlogit[slot][tid];
            const bf16 hi = __float2bfloat16_rn(dl);
            const bf16 lo = __float2bfloat16_rn(__fsub_rn(dl, __bfloat162float(hi)));
            *reinterpret_cast<bf16 *>(sm.dls + nk_off(0, part * WG_ROWS + tid)) = hi;
            *reinterpret_cast<bf16 *>(sm.dls + nk_off(1, part * WG_ROWS + tid)) = lo;
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc_after_sync();
            const uint32_t amn = idesc_of(H, 1, 1), amn16 = idesc_of(16, 1, 0);
            const uint32_t b0 = smem_addr(sm.blk[slot][0]), b1 = smem_addr(sm.blk[slot][1]);
            const uint32_t b2 = smem_addr(sm.blk[slot][2]), b3 = smem_addr(sm.blk[slot][3]);
            const uint32_t b4 = smem_addr(sm.blk[slot][4]), bx = smem_addr(sm.x[slot]);
#pragma unroll 1
            for (int kh = 0; kh < WG_ROWS / 16; ++kh) {  // 16 rows of the reduction per step
                const int ks = part * (WG_ROWS / 16) + kh;  // the step within the tile (ones, dls)
                const uint32_t acc = (u > 0 || kh > 0) ? 1u : 0u;
                const uint32_t ko = uint32_t(kh) * 4096;
                const uint64_t ones = smem_desc(sones + ks * 256, 128, 16 * 128);
                if (group == 0) {
                    const uint64_t du = smem_desc(b0 + ko, 2048, 128);
                    tc_mma_d(tmem, du, smem_desc(b1 + ko, 2048, 128), amn, acc);        // dW4[:, 0:128]
                    tc_mma_d(tmem + 128, du, smem_desc(b2 + ko, 2048, 128), amn, acc);  // dW4[:, 128:256]
                    tc_mma_d(tmem + 256, du, ones, amn16, acc);                          // b4
                    tc_mma_d(tmem + 272, smem_desc(b3 + ko, 2048, 128), smem_desc(sdls + ks * 256, 128, 16 * 128), amn16,
                             acc);                                                       // w5 (two parts)
                } else {
                    const uint64_t da3 = smem_desc(b0 + ko, 2048, 128), da2 = smem_desc(b2 + ko, 2048, 128);
                    const uint64_t da1 = smem_desc(b4 + ko, 2048, 128);
                    tc_mma_d(tmem, da3, smem_desc(b1 + ko, 2048, 128), amn, acc);        // dW3
                    tc_mma_d(tmem + 128, da2, smem_desc(b3 + ko, 2048, 128), amn, acc);  // dW2
                    tc_mma_d(tmem + 256, da1, smem_desc(bx + kh * 512, 256, 128), idesc_of(16, 1, 1), acc);  // dW1
                    tc_mma_d(tmem + 272, da3, ones, amn16, acc);                          // b3
                    tc_mma_d(tmem + 288, da2, ones, amn16, acc);                          // b2
                    tc_mma_d(tmem + 304, da1, ones, amn16, acc);                          // b1
                }
            }
            tc_commit(&sm.mbar_mma[slot]);
        }
        done_q = u + 1;
        if (*abort_flag) break;
    }
    // the last product, then this block's partial sums, one output row per thread
    bool ok = !*abort_flag;
    const int last = (done_q + WG_SLOTS - 1) % WG_SLOTS;
    if (ok && done_q > 0) ok = wait_slot(&sm.mbar_mma[last], mma_bits, last);
    else if (tid == 0 && done_q > 0)  // given up: let the products already issued finish (bounded)
        mbar_wait(&sm.mbar_mma[last], (mma_bits >> last) & 1u, a.wait_ns);
    for (int i = 0; i < WG_SLOTS; ++i)
        if (tid == 0 && ((pend_bits >> i) & 1u)) mbar_wait(&sm.mbar_in[i], (pend_par >> i) & 1u, a.wait_ns);
    if (ok && done_q == n_q && n_q > 0) {
        const int j = (warp & 3) * 32 + (tid & 31);
        const uint32_t tl = tmem + (uint32_t((warp & 3) * 32) << 16);
        float *part = a.partial + (size_t(group) * a.wgroups + cta) * N_PARAMS;
        uint32_t r[32];
        if (group == 0) {
            for (int c = 0; c < 2 * H; c += 32) {
                tmem_ld32(r, tl + c);
                for (int q = 0; q < 32; ++q) part[OFF_W4 + (c + q) * H + j] = __uint_as_float(r[q]);
            }
            tmem_ld32(r, tl + 256);
            part[OFF_B4 + j] = __uint_as_float(r[0]);
            part[OFF_W5 + j] = __fadd_rn(__uint_as_float(r[16]), __uint_as_float(r[17]));
        } else {
            for (int c = 0; c < H; c += 32) {
                tmem_ld32(r, tl + c);
                for (int q = 0; q < 32; ++q) part[OFF_W3 + (c + q) * H + j] = __uint_as_float(r[q]);
                tmem_ld32(r, tl + 128 + c);
                for (int q = 0; q < 32; ++q) part[OFF_W2 + (c + q) * H + j] = __uint_as_float(r[q]);
            }
            tmem_ld32(r, tl + 256);
            for (int q = 0; q < KIN; ++q) part[OFF_W1 + q * H + j] = __uint_as_float(r[q]);
            part[OFF_B3 + j] = __uint_as_float(r[16]);
            tmem_ld32(r, tl + 288);
            part[OFF_B2 + j] = __uint_as_float(r[0]);
            part[OFF_B1 + j] = __uint_as_float(r[16]);
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base), "r"(4 * H) : "memory");
    }
}

// The blocks' partial sums store each weight matrix column by column (element (j, k) of an
// [H][K] matrix at k * H + j), so that the thread of output row j writes consecutive rows of a
// column together; vectors are stored as they are.  Flat parameter index of stored index s:
__device__ __forceinline__ int param_of_stored(int s)
{
    int off, K;
    if (s < OFF_B1) off = OFF_W1, K = KIN;
    else if (s >= OFF_W2 && s < OFF_B2) off = OFF_W2, K = H;
    else if (s >= OFF_W3 && s < OFF_B3) off = OFF_W3, K = H;
    else if (s >= OFF_W4 && s < OFF_B4) off = OFF_W4, K = 2 * H;
    else return s;
    const int e = s - off;
    return off + (e % H) * K + e / H;
}

// gradient = sum over the owning group's blocks of their partials, in block order (b5 is
// accumulated by the chain kernel and left alone); reads in stored order, writes by parameter
// The b5 gradient: the tiles' sums of d loss / d logit added in tile order (deterministic).
__device__ float b5_gradient(const float *b5_part, int n_tiles)
{
    float g = 0.0f;
    for (int i = 0; i < n_tiles; ++i) g += b5_part[i];
    return g;
}

__global__ void sg_reduce_grad(float *grad, const float *partial, int wgroups, const float *b5_part, int n_tiles)
{
    pdl_enter();
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si == OFF_B5) grad[OFF_B5] = b5_gradient(b5_part, n_tiles);
    if (si >= N_PARAMS || si == OFF_B5) return;
    const int group = (si >= OFF_W4 && si < OFF_B5) ? 0 : 1;
    const float *src = partial + size_t(group) * wgroups * N_PARAMS + si;
    float s = 0.0f;
    for (int c = 0; c < wgroups; ++c) s += src[size_t(c) * N_PARAMS];
    grad[param_of_stored(si)] = s;
}

// ------------------------------------------------------------------ optimizer

// position of flat parameter i in the canonical bfloat16 image of W1..W4 (-1: not a matrix weight)
__device__ __forceinline__ int canon_index(int i)
{
    int base, k_dim, j;
    if (i < OFF_B1) {
        base = WC_W1, k_dim = KIN, j = i - OFF_W1;
    } else if (i >= OFF_W2 && i < OFF_B2) {
        base = WC_W2, k_dim = H, j = i - OFF_W2;
    } else if (i >= OFF_W3 && i < OFF_B3) {
        base = WC_W3, k_dim = H, j = i - OFF_W3;
    } else if (i >= OFF_W4 && i < OFF_B4) {
        base = WC_W4, k_dim = 2 * H, j = i - OFF_W4;
    } else {
        return -1;
    }
    const int n = j / k_dim, k = j - n * k_dim;
    return base + int(canon_off(n, k, k_dim) / 2);
}

// Adam step of one step's hyper-parameters (c1, c2: the bias corrections 1 - beta^t)
struct AdamStep {
    float lr, b1, b2, eps, wd, c1, c2;
};

// Adam (with decoupled weight decay) on parameter i with gradient gi; refreshes the bfloat16
// copy and the canonical image
__device__ __forceinline__ void adam_apply(int i, float gi, float *w, float *m, float *v, bf16 *wb, bf16 *wc,
                                           const AdamStep &h)
{
    const float mi = h.b1 * m[i] + (1.0f - h.b1) * gi;
    const float vi = h.b2 * v[i] + (1.0f - h.b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / h.c1, vh = vi / h.c2;
    const float wi = w[i] - h.lr * (mh / (sqrtf(vh) + h.eps) + h.wd * w[i]);
    w[i] = wi;
    const bf16 hb = __float2bfloat16_rn(wi);
    wb[i] = hb;
    const int ci = canon_index(i);
    if (ci >= 0) wc[ci] = hb;
}

// sg_reduce_grad and the Adam step in one pass (a training step).  Each weight matrix is cut
// into 16 x 16 tiles, one 256-thread block per tile: thread (x, y) first sums, over the blocks'
// partials in block order, stored element (row j0 + x, column k0 + y) (reads along rows, the
// stored order), the tile goes through shared memory, and thread (x, y) then applies Adam to
// parameter (row j0 + y, column k0 + x) (parameter order).  The vectors (biases, w5) follow in
// blocks of their own; b5's gradient is the chain kernel's.
constexpr int RA_TILES_W1 = (H / 16) * (KIN / 16), RA_TILES_W2 = (H / 16) * (H / 16);
constexpr int RA_TILES_W4 = (H / 16) * (2 * H / 16);
constexpr int RA_MATRIX_BLOCKS = RA_TILES_W1 + 2 * RA_TILES_W2 + RA_TILES_W4;
constexpr int RA_VECTOR_BLOCKS = (5 * H + 1 + 255) / 256;  // b1, b2, b3, b4, w5, b5

__global__ void __launch_bounds__(256) sg_reduce_adam(float *grad, const float *partial, int wgroups, float *w,
                                                      float *m, float *v, bf16 *wb, bf16 *wc, AdamStep h,
                                                      const float *b5_part, int n_tiles)
{
    pdl_enter();
    __shared__ float tile[16][17];
    const int tid = threadIdx.x;
    int blk = blockIdx.x;
    if (blk >= RA_MATRIX_BLOCKS) {
        const int e = (blk - RA_MATRIX_BLOCKS) * 256 + tid;  // index among the vector parameters
        if (e > 5 * H) return;
        int pidx;
        if (e == 5 * H) pidx = OFF_B5;
        else {
            const int which = e / H, r = e % H;
            const int offs[5] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4, OFF_W5};
            pidx = offs[which] + r;
        }
        float g;
        if (pidx == OFF_B5) {
            g = b5_gradient(b5_part, n_tiles);
            grad[OFF_B5] = g;
        } else {
            const int group = pidx >= OFF_W4 ? 0 : 1;
            const float *src = partial + size_t(group) * wgroups * N_PARAMS + pidx;
            g = 0.0f;
            for (int c = 0; c < wgroups; ++c) g += src[size_t(c) * N_PARAMS];
            grad[pidx] = g;
        }
        adam_apply(pidx, g, w, m, v, wb, wc, h);
        return;
    }
    int off, K, group;
    if (blk < RA_TILES_W1) off = OFF_W1, K = KIN, group = 1;
    else if ((blk -= RA_TILES_W1) < RA_TILES_W2) off = OFF_W2, K = H, group = 1;
    else if ((blk -= RA_TILES_W2) < RA_TILES_W2) off = OFF_W3, K = H, group = 1;
    else blk -= RA_TILES_W2, off = OFF_W4, K = 2 * H, group = 0;
    const int kt = K / 16;
    const int j0 = (blk / kt) * 16, k0 = (blk % kt) * 16;
    const int x = tid & 15, y = tid >> 4;
    {
        const int si = off + (k0 + y) * H + (j0 + x);  // stored: column k0 + y, row j0 + x
        const float *src = partial + size_t(group) * wgroups * N_PARAMS + si;
        float g = 0.0f;
        for (int c = 0; c < wgroups; ++c) g += src[size_t(c) * N_PARAMS];
        tile[y][x] = g;
    }
    __syncthreads();
    const float g = tile[x][y];                           // row j0 + y, column k0 + x
    const int pidx = off + (j0 + y) * K + (k0 + x);
    grad[pidx] = g;
    adam_apply(pidx, g, w, m, v, wb, wc, h);
}

__global__ void sg_to_bf16(const float *w, bf16 *wb, bf16 *wc, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bf16 h = __float2bfloat16_rn(w[i]);
    wb[i] = h;
    const int ci = canon_index(i);
    if (ci >= 0) wc[ci] = h;
}

// bbe_surrogate_wait_probe: one warp waits, with the surrogate kernels' bounded wait, on an
// mbarrier that no thread arrives at and no copy completes; the wait gives up after limit_ns and
// the warp records it in the status word, as the surrogate kernels do.  Nothing is in flight
// when it gives up (no copy, no tensor-core operation, no tensor memory).
__global__ void sg_wait_probe(int *status, long long limit_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool done = __all_sync(0xffffffffu, mbar_wait(&bar, 0u, limit_ns));
    if (!done && threadIdx.x == 0) atomicOr(status, 1);
}

__global__ void scatter_probs(const float *src, const int32_t *dst_index, float *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[dst_index[i]] = src[i];
}

// Monte Carlo fallback: probability of sub-batch competitor i = its count over its race's
// total budget, written to competitor dst[i] of the query batch (the division of bbe_win_probs)
__global__ void fallback_probs(const int32_t *counts, const int32_t *comp_race, const int64_t *total,
                               const int32_t *dst, float *probs, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) probs[dst[i]] = __fdiv_rn(__int2float_rn(counts[i]), __ll2float_rn(total[comp_race[i]]));
}

// acc[map[i]] += add[i]: second-stage counts into the first stage's
__global__ void add_counts(int32_t *acc, const int32_t *add, const int32_t *map, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[map[i]] += add[i];
}

// confidence gate: flag[i] = 1 when the second-largest output probability of race races[i]
// exceeds runner_up_max
__global__ void sg_gate(const int32_t *race_off, const int32_t *races, int n, const float *probs, float runner_up_max,
                        uint8_t *flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = races[i];
    float m1 = -1.0f, m2 = -1.0f;
    for (int c = race_off[r]; c < race_off[r + 1]; ++c) {
        const float p = probs[c];
        if (p > m1) {
            m2 = m1;
            m1 = p;
        } else if (p > m2) {
            m2 = p;
        }
    }
    flag[i] = m2 > runner_up_max ? 1 : 0;
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
    bf16 *wc = nullptr;                                                // canonical W1..W4 image
    int *d_status = nullptr;                                           // bounded-wait status word
    // forward scratch: per-tile features, race layout records and logits
    unsigned char *d_xbuf = nullptr;
    size_t xbuf_cap = 0;
    TileMeta *d_meta = nullptr;
    size_t meta_cap = 0;
    float *d_logits = nullptr;
    size_t logits_cap = 0;
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
    unsigned char *ws = nullptr;  // training workspace, WS_TILE bytes per tile
    float *ws_dlogit = nullptr;
    float *ws_b5 = nullptr;       // per-tile terms of the b5 gradient
    size_t ws_tiles = 0;
    float *d_partial = nullptr;   // weight-gradient partials of the backward's blocks
    size_t partial_cap = 0;
    float *d_loss = nullptr;
    SgRanges ranges;
    uint64_t ranges_version = 1;
    // inference plan cached per (batch, ranges): network races packed into tiles, fallback races
    uint64_t iplan_serial = 0, iplan_version = 0;
    std::vector<int32_t> iplan_net;  // races the network answers (tile order)
    std::vector<int32_t> iplan_mc;   // races outside the training ranges
    std::vector<uint8_t> iplan_flag;
    // confidence gate: runner-up probability above which a race goes to Monte Carlo
    float gate = 1.0f;
    int32_t raw_only = 0;  // 1: the network sees the five raw inputs only
    uint8_t *d_gate = nullptr;
    size_t gate_cap = 0;
    // two-stage fallback (pilot 0: each race's own budget) and the last call's fallback totals
    int64_t fb_pilot = 0;
    double fb_sd = 0.0;
    int64_t fb_races = 0, fb_rollouts = 0;
    double fb_times[5] = {0, 0, 0, 0, 0};  // last fallback: staging, pilot, budget, top-up staging, top-up and finish (s)
    int64_t iplan_tiles = 0;
    SgTile *d_itiles = nullptr;
    size_t itiles_cap = 0;
    int32_t *d_iorder = nullptr;
    size_t iorder_cap = 0;
};

namespace {

size_t fwd_smem() { return sizeof(TcSmem); }
size_t chain_smem() { return sizeof(BcSmem); }
size_t wgrad_smem() { return sizeof(BwSmem); }

bbe_status ensure_attrs()
{
    static bool done = false;
    if (done) return BBE_OK;
    SG_TRY(cudaFuncSetAttribute(sg_forward_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(fwd_smem())));
    SG_TRY(cudaFuncSetAttribute(sg_forward_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(fwd_smem())));
    SG_TRY(cudaFuncSetAttribute(sg_backward_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, int(chain_smem())));
    SG_TRY(cudaFuncSetAttribute(sg_backward_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wgrad_smem())));
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
    if (s->ws_b5) cudaFree(s->ws_b5);
    s->ws = nullptr;
    s->ws_dlogit = nullptr;
    s->ws_b5 = nullptr;
    s->ws_tiles = 0;
    SG_TRY(cudaMalloc(&s->ws, tiles * WS_TILE));
    SG_TRY(cudaMalloc(&s->ws_dlogit, tiles * TILE * sizeof(float)));
    SG_TRY(cudaMalloc(&s->ws_b5, tiles * sizeof(float)));
    s->ws_tiles = tiles;
    return BBE_OK;
}

SgArgs base_args(const bbe_surrogate *s, const bbe_batch *b)
{
    SgArgs a{};
    a.wb = s->wb;
    a.wc = s->wc;
    a.wf = s->w;
    a.status = s->d_status;
    a.wait_ns = kWaitNs;
    a.b = b->dev;
    a.tiles = s->d_tiles;
    a.order = s->d_order;
    a.raw_only = s->raw_only;
    return a;
}

// The shuffled race order of training epoch e (1, 2, ...): a permutation of the batch's races
// drawn from the configuration's shuffle seed and e alone, so that a handle loaded from a
// checkpoint continues the epoch it was saved in.
void epoch_permutation(std::vector<int32_t> &order, int32_t n_races, uint64_t shuffle_seed, uint64_t e)
{
    order.resize(size_t(n_races));
    std::iota(order.begin(), order.end(), 0);
    std::mt19937_64 rng(shuffle_seed ^ (0x9E3779B97F4A7C15ull * e));
    std::shuffle(order.begin(), order.end(), rng);
}

// Launch with programmatic stream serialization: the kernel may be scheduled while the one
// before it on the stream finishes (every surrogate kernel waits for its predecessors in
// pdl_enter before it reads their results).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// forward over n_tiles tiles of a.tiles/a.order: features (one block per tile), the
// persistent tensor-core kernel (two tile pipelines per block, at most one block per SM), softmax
bbe_status launch_forward(bbe_surrogate *s, SgArgs &a, int64_t n_tiles, cudaStream_t st)
{
    if (n_tiles <= 0) return BBE_OK;
    bbe_status e;
    if ((e = ensure_buf(s->d_xbuf, s->xbuf_cap, size_t(n_tiles) * TILE * KIN * sizeof(bf16)))) return e;
    if ((e = ensure_buf(s->d_meta, s->meta_cap, size_t(n_tiles)))) return e;
    if ((e = ensure_buf(s->d_logits, s->logits_cap, size_t(n_tiles) * TILE))) return e;
    a.xbuf = s->d_xbuf;
    a.meta = s->d_meta;
    a.logits = s->d_logits;
    int dev = 0, sms = 0;
    SG_TRY(cudaGetDevice(&dev));
    SG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n_tiles + 1) / 2, sms));
    SG_TRY(launch_pdl(sg_prep, unsigned(n_tiles), TILE, 0, st, a));
    if (a.train)
        SG_TRY(launch_pdl(sg_forward_tc<true>, unsigned(grid), TC_THREADS, fwd_smem(), st, a, int(n_tiles)));
    else
        SG_TRY(launch_pdl(sg_forward_tc<false>, unsigned(grid), TC_THREADS, fwd_smem(), st, a, int(n_tiles)));
    if (a.train || !a.probs)
        SG_TRY(launch_pdl(sg_softmax, unsigned(n_tiles), TILE, 0, st, a, int(n_tiles)));
    else
        SG_TRY(launch_pdl(sg_softmax_infer, unsigned((n_tiles + 7) / 8), 256, 0, st, a, int(n_tiles)));
    return BBE_OK;
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

// every buffer a training pass of up to max_nt tiles needs, allocated before the steps are
// launched (a reallocation between launches would synchronise the device)
bbe_status ensure_train_buffers(bbe_surrogate *s, int64_t max_nt)
{
    if (max_nt <= 0) return BBE_OK;
    bbe_status e;
    int dev = 0, sms = 0;
    SG_TRY(cudaGetDevice(&dev));
    SG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if ((e = ensure_ws(s, size_t(max_nt)))) return e;
    if ((e = ensure_buf(s->d_xbuf, s->xbuf_cap, size_t(max_nt) * TILE * KIN * sizeof(bf16)))) return e;
    if ((e = ensure_buf(s->d_meta, s->meta_cap, size_t(max_nt)))) return e;
    if ((e = ensure_buf(s->d_logits, s->logits_cap, size_t(max_nt) * TILE))) return e;
    const int64_t groups = std::max<int64_t>(1, std::min<int64_t>(max_nt, std::max(1, sms / 2)));
    if ((e = ensure_buf(s->d_partial, s->partial_cap, size_t(2) * groups * N_PARAMS))) return e;
    return BBE_OK;
}

// one training pass (forward + backward) over tiles [t0, t1) of the uploaded plan
// The forward and backward passes of one step over tiles t0 .. t1-1; the gradient lands in
// s->grad, and with `adam` the parameters take the Adam step in the same final kernel.
bbe_status train_pass(bbe_surrogate *s, const bbe_batch *b, const float *target, int64_t t0, int64_t t1,
                      int64_t races, float *loss_slot, cudaStream_t st, const AdamStep *adam = nullptr)
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
    a.b5_part = s->ws_b5;
    a.train = 1;
    int dev = 0, sms = 0;
    SG_TRY(cudaGetDevice(&dev));
    SG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // weight-gradient blocks per group: every block gets at least one tile
    a.wgroups = int32_t(std::max<int64_t>(1, std::min<int64_t>(nt, std::max(1, sms / 2))));
    if ((e = ensure_buf(s->d_partial, s->partial_cap, size_t(2) * a.wgroups * N_PARAMS))) return e;
    a.partial = s->d_partial;
    if ((e = launch_forward(s, a, nt, st))) return e;
    SG_TRY(launch_pdl(sg_backward_chain, unsigned(std::min<int64_t>(nt, sms)), 256, chain_smem(), st, a, int(nt)));
    SG_TRY(launch_pdl(sg_backward_wgrad, unsigned(2 * a.wgroups), 128, wgrad_smem(), st, a, int(nt)));
    if (adam)
        SG_TRY(launch_pdl(sg_reduce_adam, unsigned(RA_MATRIX_BLOCKS + RA_VECTOR_BLOCKS), 256, 0, st, s->grad,
                          static_cast<const float *>(s->d_partial), a.wgroups, s->w, s->m, s->v, s->wb, s->wc, *adam,
                          static_cast<const float *>(s->ws_b5), int(nt)));
    else
        SG_TRY(launch_pdl(sg_reduce_grad, unsigned((N_PARAMS + 255) / 256), 256, 0, st, s->grad,
                          static_cast<const float *>(s->d_partial), a.wgroups, static_cast<const float *>(s->ws_b5),
                          int(nt)));
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
    SG_TRY(cudaMalloc(&s->wc, WC_ELEMS * sizeof(bf16)));
    SG_TRY(cudaMalloc(&s->d_status, sizeof(int)));
    SG_TRY(cudaMemset(s->d_status, 0, sizeof(int)));
    SG_TRY(cudaMalloc(&s->d_loss, sizeof(float)));
    SG_TRY(cudaMemset(s->m, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMemset(s->v, 0, N_PARAMS * sizeof(float)));
    return BBE_OK;
}

bbe_status upload_params(bbe_surrogate *s, const float *host)
{
    SG_TRY(cudaMemcpy(s->w, host, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    sg_to_bf16<<<(N_PARAMS + 255) / 256, 256>>>(s->w, s->wb, s->wc, N_PARAMS);
    SG_TRY(cudaGetLastError());
    SG_TRY(cudaMemset(s->m, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaMemset(s->v, 0, N_PARAMS * sizeof(float)));
    SG_TRY(cudaDeviceSynchronize());
    s->step = 0;
    return BBE_OK;
}

void free_surrogate(bbe_surrogate *s)
{
    for (void *p : {(void *)s->w, (void *)s->m, (void *)s->v, (void *)s->grad, (void *)s->wb, (void *)s->wc,
                    (void *)s->d_status, (void *)s->d_xbuf, (void *)s->d_meta, (void *)s->d_logits, (void *)s->d_tiles,
                    (void *)s->d_order, (void *)s->ws, (void *)s->ws_dlogit, (void *)s->ws_b5, (void *)s->d_loss, (void *)s->d_itiles,
                    (void *)s->d_iorder, (void *)s->d_gate, (void *)s->d_partial})
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
    if ((e = launch_forward(s, a, int64_t(tiles.size()), st))) return e;
    SG_TRY(bbe::note_use(b, st));
    return BBE_OK;
}

}  // namespace

namespace {

// Budget rule of the two-stage fallback (include/bbe_surrogate.h, bbe_surrogate_fallback_budget).
int64_t fallback_budget(int n, const int32_t *counts, int64_t pilot, int64_t cap, double max_sd)
{
    if (n == 1) return pilot;  // the lone competitor wins every rollout that finishes
    const double R1 = double(pilot);
    double v = 0.0;
    for (int c = 0; c < n; ++c) {
        const double p = double(counts[c]) / R1;
        const double h = 3.0 * std::sqrt(std::max(p * (1.0 - p), 1.0 / R1) / R1);
        const double q = std::min(std::max(0.5, p - h), p + h);  // nearest point to 1/2
        v = std::max(v, q * (1.0 - q));
    }
    const double need = std::ceil(v / (max_sd * max_sd));
    const int64_t r = need >= double(cap) ? cap : int64_t(need);
    return std::min(cap, std::max(pilot, r));
}

// Device buffers and batches of one fallback call, released on every exit.
struct FallbackScratch {
    std::vector<void *> mem;
    std::vector<bbe_batch *> batches;
    cudaStream_t st = nullptr;
    template <typename T>
    bbe_status alloc(T **p, size_t count)
    {
        *p = nullptr;
        if (cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
            bbe::set_error("Monte Carlo fallback: device allocation failed");
            return BBE_ERR_CUDA;
        }
        mem.push_back(*p);
        return BBE_OK;
    }
    ~FallbackScratch()
    {
        cudaStreamSynchronize(st);
        for (void *p : mem) cudaFree(p);
        for (bbe_batch *b : batches) bbe_destroy_batch(b);
    }
};

// A batch of races `races` of b with budgets R (and first rollouts k0 when not null), each
// race keeping its own stream id; src[j] = the competitor of b that competitor j copies.
bbe_status stage_subset(const bbe_batch *b, const std::vector<int32_t> &races, const std::vector<int64_t> &R,
                        const std::vector<int64_t> *k0, FallbackScratch &sc, bbe_batch **out,
                        std::vector<int32_t> &src)
{
    std::vector<int32_t> off(1, 0), ids;
    std::vector<float> L, d0, mu, sg, rho, P, th, pv;
    src.clear();
    for (int r : races) {
        const int a0 = b->h_off[r], a1 = b->h_off[r + 1];
        off.push_back(off.back() + (a1 - a0));
        L.push_back(b->h_L[r]);
        ids.push_back(b->h_race_ids.empty() ? int32_t(b->race_id0 + uint32_t(r)) : b->h_race_ids[r]);
        for (int i = a0; i < a1; ++i) {
            d0.push_back(b->h_d0[i]);
            mu.push_back(b->h_mu[i]);
            sg.push_back(b->h_sigma[i]);
            rho.push_back(b->h_rho[i]);
            P.push_back(b->h_P[i]);
            th.push_back(b->h_theta[i]);
            if (!b->h_prev.empty()) pv.push_back(b->h_prev[i]);
            src.push_back(i);
        }
    }
    bbe_batch *sub = nullptr;
    bbe_status e = bbe::stage_batch(&sub, int32_t(races.size()), off.data(), L.data(), R.data(), d0.data(),
                                    mu.data(), sg.data(), rho.data(), P.data(), th.data(),
                                    pv.empty() ? nullptr : pv.data(), b->seed, bbe_dist(b->dist), 0, ids.data(), sc.st);
    if (e) return e;
    sc.batches.push_back(sub);
    if ((e = bbe_batch_set_cfg(sub, &b->cfg))) return e;
    if (k0 && (e = bbe::set_first_rollouts(sub, k0->data()))) return e;
    *out = sub;
    return BBE_OK;
}

// Plain Monte Carlo for races `mc` of b, written into probs.  Without a pilot every race runs
// its own budget.  With one, every race first runs min(pilot, R) rollouts; the budget rule
// then sets its total from those counts, and the missing rollouts (the next indices of the
// same stream) run as a second batch whose counts are added to the first: the result is
// plain Monte Carlo at the total budget.
bbe_status mc_fallback(bbe_surrogate *s, const bbe_batch *b, const std::vector<int32_t> &mc, float *probs,
                       cudaStream_t st)
{
    FallbackScratch sc;
    sc.st = st;
    const size_t m = mc.size();
    using clk = std::chrono::steady_clock;
    auto t_mark = clk::now();
    auto lap = [&](int slot) {
        const auto now = clk::now();
        s->fb_times[slot] += std::chrono::duration<double>(now - t_mark).count();
        t_mark = now;
    };
    for (double &t : s->fb_times) t = 0.0;
    std::vector<int64_t> cap(m), R1(m);
    for (size_t i = 0; i < m; ++i) {
        cap[i] = b->h_R[size_t(mc[i])];
        R1[i] = s->fb_pilot > 0 ? std::min(s->fb_pilot, cap[i]) : cap[i];
    }
    bbe_status e;
    bbe_batch *sub1 = nullptr;
    std::vector<int32_t> dst1;
    if ((e = stage_subset(b, mc, R1, nullptr, sc, &sub1, dst1))) return e;
    lap(0);
    const size_t n1 = dst1.size();
    int32_t *c1 = nullptr, *d_dst = nullptr;
    int64_t *d_total = nullptr;
    if ((e = sc.alloc(&c1, n1)) || (e = sc.alloc(&d_dst, n1)) || (e = sc.alloc(&d_total, m))) return e;
    if ((e = bbe_rollout_batch(sub1, c1, nullptr, st))) return e;
    std::vector<int64_t> total = R1;
    if (s->fb_pilot > 0) {
        std::vector<int32_t> h1(n1);
        SG_TRY(cudaMemcpyAsync(h1.data(), c1, n1 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if ((e = bbe_batch_status(sub1, st))) return e;  // synchronises the stream
        lap(1);
        std::vector<int32_t> races2, map2;
        std::vector<int64_t> R2, k2;
        for (size_t i = 0; i < m; ++i) {
            const int a0 = sub1->h_off[i], a1 = sub1->h_off[i + 1];
            total[i] = fallback_budget(a1 - a0, h1.data() + a0, R1[i], cap[i], s->fb_sd);
            if (total[i] > R1[i]) {
                races2.push_back(mc[i]);
                R2.push_back(total[i] - R1[i]);
                k2.push_back(R1[i]);
                for (int j = a0; j < a1; ++j) map2.push_back(j);
            }
        }
        lap(2);
        if (!races2.empty()) {
            bbe_batch *sub2 = nullptr;
            std::vector<int32_t> src2;
            if ((e = stage_subset(b, races2, R2, &k2, sc, &sub2, src2))) return e;
            lap(3);
            const size_t n2 = map2.size();
            int32_t *c2 = nullptr, *d_map = nullptr;
            if ((e = sc.alloc(&c2, n2)) || (e = sc.alloc(&d_map, n2))) return e;
            SG_TRY(cudaMemcpyAsync(d_map, map2.data(), n2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            if ((e = bbe_rollout_batch(sub2, c2, nullptr, st))) return e;
            add_counts<<<unsigned((n2 + 255) / 256), 256, 0, st>>>(c1, c2, d_map, int(n2));
            SG_TRY(cudaGetLastError());
            if ((e = bbe_batch_status(sub2, st))) return e;
        }
    }
    SG_TRY(cudaMemcpyAsync(d_total, total.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SG_TRY(cudaMemcpyAsync(d_dst, dst1.data(), n1 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    fallback_probs<<<unsigned((n1 + 255) / 256), 256, 0, st>>>(c1, sub1->dev.comp_race, d_total, d_dst, probs, int(n1));
    SG_TRY(cudaGetLastError());
    if ((e = bbe_batch_status(sub1, st))) return e;  // synchronises: host vectors stay alive until here
    lap(4);
    int64_t sum = 0;
    for (int64_t t : total) sum += t;
    s->fb_rollouts = sum;
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
    if (b->dev.law != BBE_LAW_POSITION) {
        bbe::set_error("the surrogate takes position-law batches only (its inputs carry no elapsed time)");
        return BBE_ERR_UNSUPPORTED;
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
    SG_TRY(bbe::note_use(b, st));
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
    if (b->dev.law != BBE_LAW_POSITION) {
        bbe::set_error("the surrogate takes position-law batches only (its inputs carry no elapsed time)");
        return BBE_ERR_UNSUPPORTED;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    bbe_status e;
    if ((e = ensure_attrs())) return e;
    if (!s->ranges.valid) {
        record_ranges(s->ranges, b);
        s->ranges_version += 1;
    }
    if (s->plan_batch != b || int64_t(s->epoch_order.size()) != b->n_races) {
        // a handle loaded from a checkpoint (no batch seen yet, in the middle of an epoch)
        // continues that epoch; any other change of batch starts a new one
        const bool resume = s->plan_batch == nullptr && s->epoch > 0 && s->cursor > 0 && s->cursor < b->n_races;
        s->plan_batch = b;
        s->epoch_order.clear();
        if (resume) epoch_permutation(s->epoch_order, b->n_races, cfg->shuffle_seed, s->epoch);
        else s->cursor = 0;
    }
    if (loss_log) SG_TRY(cudaMemsetAsync(loss_log, 0, size_t(cfg->steps) * sizeof(float), st));
    // plan every step of the call on the host first (per-epoch shuffle, tile packing), upload
    // the plan once, then launch the steps back to back
    std::vector<int32_t> all_order;
    std::vector<SgTile> all_tiles;
    std::vector<int64_t> tile_begin(size_t(cfg->steps) + 1, 0), races_in(size_t(cfg->steps), 0);
    int64_t max_nt = 0;
    for (int32_t k = 0; k < cfg->steps; ++k) {
        if (s->epoch_order.empty() || s->cursor >= int64_t(s->epoch_order.size())) {
            s->epoch += 1;
            epoch_permutation(s->epoch_order, b->n_races, cfg->shuffle_seed, s->epoch);
            s->cursor = 0;
        }
        const int64_t take = std::min<int64_t>(cfg->batch_states, int64_t(s->epoch_order.size()) - s->cursor);
        const int64_t base = int64_t(all_order.size());
        all_order.insert(all_order.end(), s->epoch_order.begin() + s->cursor, s->epoch_order.begin() + s->cursor + take);
        s->cursor += take;
        pack_tiles(b->h_off, all_order.data() + base, take, base, all_tiles);
        tile_begin[size_t(k) + 1] = int64_t(all_tiles.size());
        races_in[size_t(k)] = take;
        max_nt = std::max<int64_t>(max_nt, tile_begin[size_t(k) + 1] - tile_begin[size_t(k)]);
    }
    if ((e = upload_plan(s, all_order, all_tiles, st))) return e;
    if ((e = ensure_train_buffers(s, max_nt))) return e;
    for (int32_t k = 0; k < cfg->steps; ++k) {
        const float t = float(s->step + 1);
        const AdamStep h{cfg->lr, cfg->beta1, cfg->beta2, cfg->eps, cfg->weight_decay,
                         1.0f - std::pow(cfg->beta1, t), 1.0f - std::pow(cfg->beta2, t)};
        if ((e = train_pass(s, b, target, tile_begin[size_t(k)], tile_begin[size_t(k) + 1], races_in[size_t(k)],
                            loss_log ? loss_log + k : nullptr, st, &h)))
            return e;
        s->step += 1;
    }
    SG_TRY(bbe::note_use(b, st));
    return BBE_OK;
}

bbe_status bbe_surrogate_forward(bbe_surrogate *s, const bbe_batch *b, float *probs, void *cuda_stream)
{
    if (!s || !b || !probs) {
        bbe::set_error("surrogate, batch or probs is NULL");
        return BBE_ERR_ARG;
    }
    if (b->dev.law != BBE_LAW_POSITION) {
        bbe::set_error("the surrogate takes position-law batches only (its inputs carry no elapsed time)");
        return BBE_ERR_UNSUPPORTED;
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
    if (b->dev.law != BBE_LAW_POSITION) {
        bbe::set_error("the surrogate takes position-law batches only (its inputs carry no elapsed time)");
        return BBE_ERR_UNSUPPORTED;
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
        s->iplan_net = std::move(net);
        s->iplan_serial = b->serial;
        s->iplan_version = s->ranges_version;
    }
    if (s->iplan_tiles > 0) {
        SgArgs a = base_args(s, b);
        a.tiles = s->d_itiles;
        a.order = s->d_iorder;
        a.probs = probs;
        a.train = 0;
        if ((e = launch_forward(s, a, s->iplan_tiles, st))) return e;
    }
    std::vector<int32_t> mc = s->iplan_mc;
    std::vector<uint8_t> flag = s->iplan_flag;
    const int64_t n_net = int64_t(s->iplan_net.size());
    if (s->gate < 0.5f && n_net > 0) {
        // races the network does not call with near-certainty go to Monte Carlo as well
        if ((e = ensure_buf(s->d_gate, s->gate_cap, size_t(n_net)))) return e;
        sg_gate<<<unsigned((n_net + 255) / 256), 256, 0, st>>>(b->dev.race_off, s->d_iorder, int(n_net), probs, s->gate,
                                                              s->d_gate);
        SG_TRY(cudaGetLastError());
        std::vector<uint8_t> g(size_t(n_net), 0);
        SG_TRY(cudaMemcpyAsync(g.data(), s->d_gate, size_t(n_net), cudaMemcpyDeviceToHost, st));
        SG_TRY(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < n_net; ++i)
            if (g[size_t(i)]) {
                mc.push_back(s->iplan_net[size_t(i)]);
                flag[size_t(s->iplan_net[size_t(i)])] = 2;
            }
    }
    s->fb_races = int64_t(mc.size());
    s->fb_rollouts = 0;
    if (!mc.empty() && (e = mc_fallback(s, b, mc, probs, st))) return e;
    SG_TRY(bbe::note_use(b, st));
    if (used_mc) {
        SG_TRY(cudaMemcpyAsync(used_mc, flag.data(), flag.size(), cudaMemcpyHostToDevice, st));
        SG_TRY(cudaStreamSynchronize(st));
    }
    return BBE_OK;
}

bbe_status bbe_surrogate_set_inputs(bbe_surrogate *s, int32_t inputs)
{
    if (!s || (inputs != BBE_SURROGATE_INPUTS_RAW && inputs != BBE_SURROGATE_INPUTS_DERIVED)) {
        bbe::set_error("bbe_surrogate_set_inputs: surrogate is NULL or inputs is not 5 or 14");
        return BBE_ERR_ARG;
    }
    s->raw_only = inputs == BBE_SURROGATE_INPUTS_RAW ? 1 : 0;
    s->iplan_serial = 0;
    return BBE_OK;
}

bbe_status bbe_surrogate_set_gate(bbe_surrogate *s, float runner_up_max)
{
    if (!s || !(runner_up_max >= 0.0f && runner_up_max <= 1.0f)) {
        bbe::set_error("bbe_surrogate_set_gate: surrogate is NULL or runner_up_max outside [0, 1]");
        return BBE_ERR_ARG;
    }
    s->gate = runner_up_max;
    return BBE_OK;
}

bbe_status bbe_surrogate_set_fallback(bbe_surrogate *s, int64_t pilot_rollouts, double max_sd)
{
    if (!s || pilot_rollouts < 0 || pilot_rollouts > INT32_MAX ||
        (pilot_rollouts > 0 && !(max_sd > 0.0 && max_sd <= 0.5))) {
        bbe::set_error("bbe_surrogate_set_fallback: surrogate is NULL, pilot_rollouts outside 0..2^31-1 or "
                       "max_sd outside (0, 0.5]");
        return BBE_ERR_ARG;
    }
    s->fb_pilot = pilot_rollouts;
    s->fb_sd = max_sd;
    return BBE_OK;
}

bbe_status bbe_surrogate_fallback_budget(int32_t n, const int32_t *counts, int64_t pilot, int64_t cap, double max_sd,
                                         int64_t *budget)
{
    if (n < 1 || !counts || !budget || pilot < 1 || cap < pilot || !(max_sd > 0.0 && max_sd <= 0.5)) {
        bbe::set_error("bbe_surrogate_fallback_budget: n < 1, NULL pointer, pilot < 1, cap < pilot or max_sd "
                       "outside (0, 0.5]");
        return BBE_ERR_ARG;
    }
    *budget = fallback_budget(n, counts, pilot, cap, max_sd);
    return BBE_OK;
}

bbe_status bbe_surrogate_fallback_times(const bbe_surrogate *s, double *seconds)
{
    if (!s || !seconds) {
        bbe::set_error("surrogate or seconds is NULL");
        return BBE_ERR_ARG;
    }
    for (int i = 0; i < 5; ++i) seconds[i] = s->fb_times[i];
    return BBE_OK;
}

bbe_status bbe_surrogate_fallback_stats(const bbe_surrogate *s, int64_t *races, int64_t *rollouts)
{
    if (!s) {
        bbe::set_error("surrogate is NULL");
        return BBE_ERR_ARG;
    }
    if (races) *races = s->fb_races;
    if (rollouts) *rollouts = s->fb_rollouts;
    return BBE_OK;
}

bbe_status bbe_surrogate_wait_probe(bbe_surrogate *s, int64_t limit_ns, void *cuda_stream)
{
    if (!s || limit_ns < 0 || limit_ns > kWaitNs) {
        bbe::set_error("bbe_surrogate_wait_probe: surrogate is NULL or limit_ns outside 0 .. 2e9");
        return BBE_ERR_ARG;
    }
    sg_wait_probe<<<1, 32, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(s->d_status, (long long)limit_ns);
    SG_TRY(cudaGetLastError());
    return BBE_OK;
}

bbe_status bbe_surrogate_status(bbe_surrogate *s, void *cuda_stream)
{
    if (!s) {
        bbe::set_error("surrogate is NULL");
        return BBE_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int h = 0;
    SG_TRY(cudaStreamSynchronize(st));
    SG_TRY(cudaMemcpy(&h, s->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        SG_TRY(cudaMemset(s->d_status, 0, sizeof(int)));
        bbe::set_error("a surrogate kernel gave up a bounded device wait");
        return BBE_ERR_TIMEOUT;
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
    const char magic[8] = {'B', 'B', 'E', 'S', 'G', '0', '0', '2'};
    const int64_t n = N_PARAMS;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
              std::fwrite(&s->raw_only, 4, 1, f) == 1 &&
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
    int32_t raw_only = 0;
    // version 2 adds the input mode after the parameter count; version 1 files are read too
    bool ok = std::fread(magic, 1, 8, f) == 8 &&
              (std::memcmp(magic, "BBESG001", 8) == 0 || std::memcmp(magic, "BBESG002", 8) == 0) &&
              std::fread(&n, 8, 1, f) == 1 && n == N_PARAMS &&
              (magic[7] == '1' || std::fread(&raw_only, 4, 1, f) == 1) && std::fread(&step, 8, 1, f) == 1 &&
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
    s->raw_only = raw_only ? 1 : 0;
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
