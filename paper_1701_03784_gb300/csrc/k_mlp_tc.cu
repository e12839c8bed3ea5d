// Surrogate network inference on the 5th-generation tensor cores: BF16 operands in shared
// memory, FP32 accumulation in tensor memory (TMEM).
//
// One CTA takes two tiles of 128 samples of one ensemble member through every layer, in
// ping-pong: while the tensor cores run one tile's products of a layer, the other tile's
// epilogue of its previous layer runs on the CUDA cores.
//  * the activations of each tile (128 x K) sit in shared memory in the no-swizzle
//    K-major layout (8 x 8 core matrices of 16-byte rows, K-adjacent core matrices 128
//    bytes apart, 8-row groups K/8 x 128 bytes apart); the layer's weights stream through
//    a 64 KB buffer in chunks of all its output rows (at most 256) by 128 of K, each one
//    contiguous run of the packed weights (chunk_off) brought by one bulk copy from the
//    load warp as soon as the products that read the buffer have completed;
//  * one thread of the control warp issues tcgen05.mma (kind::f16, M = 128, N = the layer's
//    width, 16 of K at a time) for both tiles on each chunk (the weights are read from L2
//    once per block) into the tile's 128 x 256 FP32 accumulator in TMEM (the two
//    accumulators fill TMEM's 512 columns), releasing the weight buffer with a commit and
//    signalling the tile's epilogue with another after its layer's last chunk.  Products
//    of the full width read each operand row once per layer and ask less shared-memory
//    bandwidth per flop than narrower ones (measured: N = 128 products, or chunks of 64 or
//    32 of K in a deeper ring, ran 4% to 17% slower);
//  * eight warps per tile (two per TMEM lane quadrant, each half the columns) read the
//    accumulator with tcgen05.ld, add the bias, apply the tanh-GELU (hidden layers) and
//    write the next layer's BF16 operand back into the tile, or write the FP32 outputs,
//    then tell the control thread that the tile is ready for its next layer.
// The layer-0 operand is built by the epilogue warps from the FP32 queries.  Every
// mbarrier wait is bounded (timeout counted; the block then drains what it issued and
// still frees TMEM).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstddef>

#include "pic_internal.h"

namespace pic {

namespace {
constexpr int TM = 128;       // samples per tile = MMA M
constexpr int NTILE = 2;      // tiles per CTA (ping-pong)
constexpr int EPI_WARPS = 8;  // per tile: two per TMEM lane quadrant, each half the columns
constexpr int PARTS = EPI_WARPS / 4;   // column parts per lane quadrant
constexpr int CTRL_WARP = NTILE * EPI_WARPS;   // lane 0 issues the products
constexpr int LOAD_WARP = CTRL_WARP + 1;       // lane 0 streams the weights
constexpr int NTH = (LOAD_WARP + 1) * 32;
constexpr int KMAX = 256;
constexpr int NMAX = 256;
constexpr int WROWS = 256;    // output rows per weight chunk (N of each product)
constexpr int WK = 128;       // K columns per weight chunk
constexpr int NBUF = 1;       // weight buffers
constexpr int TMEM_COLS = 512;    // training products
constexpr int MIN_BLOCKS = 1;     // inference blocks resident per SM
constexpr int INF_TMEM = NTILE * 256;   // inference accumulators: 256 columns a tile
constexpr int BIAS_MAX = MLP_MAX_LAYERS * NMAX;
constexpr long long WAIT_LIMIT = 1LL << 22;

struct PingSmem {
    uint16_t a[NTILE][TM * KMAX];        // activations of each tile, core-matrix layout
    uint16_t w[NBUF][WROWS * WK];        // weight chunks: 128 output rows x 128 of K
    alignas(16) float bias[BIAS_MAX];    // every layer's bias of the member (bmember used)
    unsigned long long wfull[NBUF];      // a weight buffer landed
    unsigned long long wempty[NBUF];     // the products that read a weight buffer completed
    unsigned long long accdone[NTILE];   // a tile's products of a layer completed
    unsigned long long ready[NTILE];     // a tile's operand for its next layer is written
    unsigned long long bbar;             // the biases landed
    unsigned int tmem;
};
static_assert(offsetof(PingSmem, w) % 1024 == 0 && offsetof(PingSmem, bias) % 16 == 0,
              "bulk-copy destinations and operand tiles must stay aligned");

// element offset of (row r, column k) in a core-matrix tile with kp (padded) columns
__host__ __device__ __forceinline__ int core_off(int r, int k, int kp) {
    return ((r >> 3) * (kp >> 3) * 64) + ((k >> 3) * 64) + ((r & 7) * 8) + (k & 7);
}

// element offset of weight (row r, column k) of a layer's packed np x kp weights: chunk
// (q, kc) = rows [128 q, ...) x columns [128 kc, ...) is one contiguous run (the rows of
// every earlier row slice, then this slice's earlier K chunks), in core-matrix layout
// with its own width, so that one bulk copy brings a chunk into shared memory
__host__ __device__ __forceinline__ long long chunk_off(int r, int k, int kp, int np) {
    const int q = r / WROWS, kc = k / WK;
    const int rows = min(WROWS, np - q * WROWS), kw = min(WK, kp - kc * WK);
    return (long long)q * WROWS * kp + (long long)rows * kc * WK +
           core_off(r - q * WROWS, k - kc * WK, kw);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) |
           ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ULL << 46);
}
// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N and M = 128
__device__ __forceinline__ unsigned idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) |
           ((unsigned)(TM >> 4) << 24);
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(unsigned d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
// 16 consecutive FP32 columns of this thread's TMEM lane, issued without waiting: the
// registers are valid after tmem_wait16 on them (which waits for every load in flight)
__device__ __forceinline__ void tmem_issue16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(unsigned (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity,
                                          long long polls = WAIT_LIMIT) {
    for (long long k = 0; k < polls; k++) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// 1-D bulk copy global -> shared completing on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
// 8 values as 8 BF16 in one 16-byte word, two per conversion (element 0 lowest)
__device__ __forceinline__ unsigned bf16x2_bits(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ uint4 pack8x2(const float *v) {
    uint4 q;
    q.x = bf16x2_bits(v[0], v[1]);
    q.y = bf16x2_bits(v[2], v[3]);
    q.z = bf16x2_bits(v[4], v[5]);
    q.w = bf16x2_bits(v[6], v[7]);
    return q;
}

// Packed pairs of FP32 (element 0 in the low half): the bias is added two columns per
// instruction on the FP32 pipes.
__device__ __forceinline__ unsigned long long f2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(unsigned long long r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// tanh-GELU of a pair, returned as two BF16 (element 0 low): 0.5 z (1 + tanh(w)),
// w = z (c0 + c1 z^2), c0 = sqrt(2/pi), c1 = 0.044715 sqrt(2/pi).  z is rounded to BF16
// once and the rest runs on BF16 pairs (the hardware tanh approximation included): the
// result is the next layer's BF16 operand, and the BF16 steps add about one rounding of
// it (relative 2^-8) to the one it takes anyway.
__device__ __forceinline__ unsigned gelu2_bf16(unsigned long long z) {
    float z0, z1;
    f2_split(z, z0, z1);
    unsigned zb, u, q, w, t, h, y;
    const unsigned c1 = 0x3D123D12u;   // BF16 pair of 0.044715 sqrt(2/pi) = 0.035677
    const unsigned c0 = 0x3F4C3F4Cu;   // BF16 pair of sqrt(2/pi) = 0.79788
    const unsigned half = 0x3F003F00u; // BF16 pair of 0.5
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(zb) : "f"(z1), "f"(z0));
    asm("mul.rn.bf16x2 %0, %1, %1;" : "=r"(u) : "r"(zb));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(q) : "r"(u), "r"(c1), "r"(c0));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(w) : "r"(zb), "r"(q));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(w));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(h) : "r"(zb), "r"(half));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(y) : "r"(h), "r"(t), "r"(h));
    return y;
}

// bias, GELU and BF16 of 16 accumulator columns c .. c+15 of row erow, written as the
// next layer's operand (core-matrix layout, np columns)
__device__ __forceinline__ void gelu_chunk(const unsigned (&r)[16], const float *bias, int c,
                                           uint16_t *act, int erow, int np) {
    const ulonglong2 *bias4 = reinterpret_cast<const ulonglong2 *>(bias + c);
    unsigned p[8];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const ulonglong2 b = bias4[j];
        p[2 * j] = gelu2_bf16(add2(f2(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1])), b.x));
        p[2 * j + 1] = gelu2_bf16(
            add2(f2(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3])), b.y));
    }
    *reinterpret_cast<uint4 *>(act + core_off(erow, c, np)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4 *>(act + core_off(erow, c + 8, np)) = make_uint4(p[4], p[5], p[6], p[7]);
}

__device__ __forceinline__ void arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// The weight chunks in the order the products use them: layer by layer, row slice q
// (output rows [128 q, 128 q + 128)), K chunk kc (columns [128 kc, 128 kc + 128)); both
// tiles' products read a chunk before the next one is needed, so each chunk is loaded
// once per block.
struct ChunkIter {
    int l = 0, q = 0, kc = 0;
    __device__ __forceinline__ bool next(const MlpTc &tc) {
        if (++kc * WK < tc.kp[l]) return true;
        kc = 0;
        if (++q * WROWS < tc.np[l]) return true;
        q = 0;
        return ++l < tc.L;
    }
    __device__ __forceinline__ bool last_of_layer(const MlpTc &tc) const {
        return (q + 1) * WROWS >= tc.np[l] && (kc + 1) * WK >= tc.kp[l];
    }
};

__global__ void __launch_bounds__(NTH, MIN_BLOCKS) k_mlp_tc(MlpTc tc, const float *X, float *Y,
                                                   long long n, long long row_base) {
    extern __shared__ unsigned char raw[];
    const unsigned pad = (1024u - (smem_u32(raw) & 1023u)) & 1023u;
    PingSmem &sm = *reinterpret_cast<PingSmem *>(raw + pad);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // members run fastest along x, so that the blocks resident at one time read the
    // weights of every member rather than all the same member's (the same lines)
    const int z = blockIdx.x;
    const long long pair0 = row_base + (long long)blockIdx.y * (NTILE * TM);
    const long long polls = tc.wait_polls;

    if (tid == 0) {
        for (int b = 0; b < NBUF; b++) {
            mbar_init(&sm.wfull[b], 1);
            mbar_init(&sm.wempty[b], 1);
        }
        for (int t = 0; t < NTILE; t++) {
            mbar_init(&sm.accdone[t], 1);
            mbar_init(&sm.ready[t], EPI_WARPS);
        }
        mbar_init(&sm.bbar, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(INF_TMEM) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = sm.tmem;
    bool ok = true;

    if (warp == LOAD_WARP) {
        // ---- weights (and once, the biases) ------------------------------------------
        if (lane == 0) {
            const unsigned bb = (unsigned)(tc.bmember * 4);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(smem_u32(&sm.bbar)), "r"(bb) : "memory");
            bulk_load(sm.bias, tc.b + (long long)z * tc.bmember, bb, &sm.bbar);
            ChunkIter it;
            long long c = 0;
            do {
                const int b = (int)(c % NBUF);
                // the products that read this buffer NBUF chunks ago have completed
                if (c >= NBUF &&
                    !mbar_wait(&sm.wempty[b], (unsigned)(((c - NBUF) / NBUF) & 1), polls)) {
                    ok = false;
                    break;
                }
                const int kp = tc.kp[it.l];
                const int rows = min(WROWS, tc.np[it.l] - it.q * WROWS);
                const int kw = min(WK, kp - it.kc * WK);
                const unsigned wb = (unsigned)(rows * kw * 2);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(smem_u32(&sm.wfull[b])), "r"(wb) : "memory");
                // the chunk is one contiguous run of the packed weights (chunk_off)
                const uint16_t *src = tc.w + (long long)z * tc.wmember + tc.woff[it.l] +
                                      chunk_off(it.q * WROWS, it.kc * WK, kp, tc.np[it.l]);
                bulk_load(sm.w[b], src, wb, &sm.wfull[b]);
                c++;
            } while (it.next(tc));
            // before the block exits, every copy issued here has landed
            const long long last = c;
            for (long long k = last > NBUF ? last - NBUF : 0; k < last; k++)
                mbar_wait(&sm.wfull[k % NBUF], (unsigned)((k / NBUF) & 1));
            mbar_wait(&sm.bbar, 0);
        }
    } else if (warp == CTRL_WARP) {
        // ---- products --------------------------------------------------------------------
        if (lane == 0) {
            ChunkIter it;
            long long c = 0;
            bool first = true;
            do {
                const int l = it.l, kp = tc.kp[l];
                const int b = (int)(c % NBUF);
                if (!mbar_wait(&sm.wfull[b], (unsigned)((c / NBUF) & 1), polls)) {
                    ok = false;
                    break;
                }
                const int rows = min(WROWS, tc.np[l] - it.q * WROWS);
                const int kw = min(WK, kp - it.kc * WK);
                const bool last_chunk = it.last_of_layer(tc);
                const unsigned w0 = smem_u32(sm.w[b]);
                const unsigned sbo_a = (unsigned)kp / 8u * 128u;
                const unsigned sbo_w = (unsigned)kw / 8u * 128u;
                const unsigned id = idesc_bf16(rows);
                for (int t = 0; t < NTILE && ok; t++) {
                    // a tile's first chunk of a layer waits for its operand (and for its
                    // accumulator to have been read)
                    if (it.q == 0 && it.kc == 0 &&
                        !mbar_wait(&sm.ready[t], (unsigned)(l & 1), polls)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const unsigned a0 = smem_u32(sm.a[t]) + (unsigned)(it.kc * (WK / 16)) * 256u;
                    const unsigned d = tmem + (unsigned)(t * 256 + it.q * WROWS);
                    for (int kk = 0; kk < kw / 16; kk++)
                        mma_bf16(d, sdesc(a0 + kk * 256u, 128u, sbo_a),
                                 sdesc(w0 + kk * 256u, 128u, sbo_w), id, it.kc > 0 || kk > 0);
                    if (last_chunk) mma_commit(&sm.accdone[t]);
                    first = false;
                }
                if (!ok) break;
                mma_commit(&sm.wempty[b]);
                c++;
            } while (it.next(tc));
            // the products in flight complete before the block frees TMEM
            if (!first) {
                mma_commit(&sm.wempty[c % NBUF]);
                mbar_wait(&sm.wempty[c % NBUF], (unsigned)((c / NBUF) & 1));
            }
        }
    } else {
        // ---- epilogues: warps 8t .. 8t+7 own tile t ----------------------------------------
        const int t = warp / EPI_WARPS, w = warp % EPI_WARPS;
        const int quad = w & 3, part = w >> 2;
        const int erow = quad * 32 + lane;
        const long long row = pair0 + (long long)t * TM + erow;
        uint16_t *act = sm.a[t];
        // layer-0 operand: the two warps of a quadrant split its 32 rows' columns
        {
            const int k0 = tc.k[0], kp = tc.kp[0];
            for (int cc = part * 8; cc < kp; cc += 8 * PARTS) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int kk = cc + j;
                    v[j] = row < n && kk < k0 ? X[row * k0 + kk] : 0.f;
                }
                *reinterpret_cast<uint4 *>(act + core_off(erow, cc, kp)) = pack8x2(v);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) arrive(&sm.ready[t]);
        ok = mbar_wait(&sm.bbar, 0, polls);
        for (int l = 0; l < tc.L && ok; l++) {
            const int np = tc.np[l];
            const bool last = l == tc.L - 1;
            if (!mbar_wait(&sm.accdone[t], (unsigned)(l & 1), polls)) {
                ok = false;
                break;
            }
            fence_after();
            const float *bias = sm.bias + tc.boff[l];
            // this warp's 16-column chunks: part p of PARTS (rounded so that two parts
            // split an odd count with the larger share first)
            const int chunks = np / 16;
            const int c0 = (chunks * part + PARTS - 1) / PARTS;
            const int c1 = (chunks * (part + 1) + PARTS - 1) / PARTS;
            const unsigned lane_base = tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(t * 256);
            if (!last && c0 < c1) {
                // hidden layer: the next chunk's TMEM load is in flight while this one is
                // computed (two register sets, alternating)
                unsigned ra[16], rb[16];
                tmem_issue16(lane_base + (unsigned)(c0 * 16), ra);
                tmem_wait16(ra);
                for (int ch = c0; ch < c1; ch += 2) {
                    if (ch + 1 < c1) tmem_issue16(lane_base + (unsigned)((ch + 1) * 16), rb);
                    gelu_chunk(ra, bias, ch * 16, act, erow, np);
                    if (ch + 1 >= c1) break;
                    tmem_wait16(rb);
                    if (ch + 2 < c1) tmem_issue16(lane_base + (unsigned)((ch + 2) * 16), ra);
                    gelu_chunk(rb, bias, (ch + 1) * 16, act, erow, np);
                    if (ch + 2 < c1) tmem_wait16(ra);
                }
            }
            for (int ch = last ? c0 : c1; ch < c1; ch++) {
                const int c = ch * 16;
                float v[16];
                tmem_ld16(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(t * 256 + c), v);
                if (row < n) {
                    const int nout = tc.n[l];
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] += bias[c + j];
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (c + j < nout) Y[((long long)z * n + row) * nout + c + j] = v[j];
                }
            }
            if (!last) {
                // the operand is written and the accumulator read: the tile's next layer
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) arrive(&sm.ready[t]);
            }
        }
    }
    if (!ok) atomicAdd(tc.err, 1u);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(INF_TMEM) : "memory");
}

// ---- products of the training path ----
// Operand packing (many blocks per product): element (r, c) of the logical R x Cc matrix at
// src[r sR + c sC] (member stride sz) -> BF16 at core_off(r, c, Cp) of an Rp x Cp tile,
// zero-padded.  The index along which the source is contiguous runs fastest.
__global__ void k_tc_pack_op(const float *src, long long sz, int sR, int sC, int R, int Cc,
                             int Rp, int Cp, uint16_t *dst, long long dz) {
    const int z = blockIdx.y;
    const float *a = src + (long long)z * sz;
    uint16_t *d = dst + (long long)z * dz;
    const bool rows_fast = sR == 1 && sC != 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Rp * Cp; i += gridDim.x * blockDim.x) {
        const int r = rows_fast ? i % Rp : i / Cp, c = rows_fast ? i / Rp : i % Cp;
        d[core_off(r, c, Cp)] =
            bf16_bits(r < R && c < Cc ? a[(long long)r * sR + (long long)c * sC] : 0.f);
    }
}

struct GemmSmem {
    uint16_t a[TM * KMAX];     // 128 rows of A, core-matrix layout
    uint16_t b[NMAX * KMAX];   // all of B
    unsigned long long mbar;   // products done
    unsigned long long lbar;   // operands landed
    unsigned int tmem;
};

struct TcGemmDev {
    const uint16_t *A, *B;     // packed operands
    long long sA, sB;          // their member strides (elements)
    float *C;
    long long sC;
    int ldc, M, N, Kp, Np, accumulate;
    unsigned int *err;
};

// One CTA: rows [128 x, 128 x + 128) of member y.  One thread brings both packed operands
// in with bulk copies and issues the products into TMEM; the four warps read their lane
// quadrants and write (or add to) C.
__global__ void __launch_bounds__(TM, 1) k_tc_gemm(TcGemmDev g) {
    extern __shared__ unsigned char raw[];
    const unsigned pad = (1024u - (smem_u32(raw) & 1023u)) & 1023u;
    GemmSmem &sm = *reinterpret_cast<GemmSmem *>(raw + pad);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.y, m0 = blockIdx.x * TM;
    if (tid == 0) {
        mbar_init(&sm.mbar, 1);
        mbar_init(&sm.lbar, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = sm.tmem;
    if (tid == 0) {
        const unsigned ab = (unsigned)(TM * g.Kp * 2), bb = (unsigned)(g.Np * g.Kp * 2);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(smem_u32(&sm.lbar)), "r"(ab + bb) : "memory");
        bulk_load(sm.a, g.A + (long long)z * g.sA + (long long)m0 * g.Kp, ab, &sm.lbar);
        bulk_load(sm.b, g.B + (long long)z * g.sB, bb, &sm.lbar);
    }
    bool ok = __syncthreads_and(mbar_wait(&sm.lbar, 0u));
    if (ok) {
        if (tid == 0) {
            fence_after();
            const unsigned a0 = smem_u32(sm.a), b0 = smem_u32(sm.b);
            const unsigned sbo = (unsigned)g.Kp / 8u * 128u;
            const unsigned id = idesc_bf16(g.Np);
            for (int kk = 0; kk < g.Kp / 16; kk++)
                mma_bf16(tmem, sdesc(a0 + kk * 256u, 128u, sbo), sdesc(b0 + kk * 256u, 128u, sbo),
                         id, kk > 0);
            mma_commit(&sm.mbar);
        }
        ok = __syncthreads_and(mbar_wait(&sm.mbar, 0u));
    }
    if (ok) {
        fence_after();
        const int m = m0 + warp * 32 + lane;
        float *c = g.C + (long long)z * g.sC + (long long)m * g.ldc;
        for (int c0 = 0; c0 < g.Np; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
            if (m < g.M) {
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (c0 + j < g.N) c[c0 + j] = g.accumulate ? c[c0 + j] + v[j] : v[j];
            }
        }
    } else {
        // a wait gave up: count it, give the copies and products in flight one more bounded
        // wait, free TMEM below
        if (tid == 0) {
            atomicAdd(g.err, 1u);
            mbar_wait(&sm.lbar, 0u);
            mbar_wait(&sm.mbar, 0u);
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS) : "memory");
}

// FP32 parameters -> BF16 core-matrix weights and FP32 biases, zero-padded
struct PackArgs {
    long long woff[MLP_MAX_LAYERS], boff[MLP_MAX_LAYERS];
};
__global__ void k_mlp_pack(MlpTc tc, const float *params, long long P, PackArgs pa) {
    const int z = blockIdx.y / tc.L, l = blockIdx.y % tc.L;
    const int kp = tc.kp[l], np = tc.np[l], k = tc.k[l], nn = tc.n[l];
    const float *W = params + (long long)z * P + pa.woff[l];
    uint16_t *dst = tc.w + (long long)z * tc.wmember + tc.woff[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np * kp; i += gridDim.x * blockDim.x) {
        const int r = i / kp, c = i % kp;
        dst[chunk_off(r, c, kp, np)] = bf16_bits(r < nn && c < k ? W[(long long)r * k + c] : 0.f);
    }
    const float *b = params + (long long)z * P + pa.boff[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        tc.b[(long long)z * tc.bmember + tc.boff[l] + i] = i < nn ? b[i] : 0.f;
}
}  // namespace

void mlp_tc_pack(const MlpTc &tc, const float *params, long long P, const long long *woff,
                 const long long *boff, cudaStream_t s) {
    PackArgs pa;
    for (int l = 0; l < tc.L; l++) {
        pa.woff[l] = woff[l];
        pa.boff[l] = boff[l];
    }
    k_mlp_pack<<<dim3(64, tc.E * tc.L), 256, 0, s>>>(tc, params, P, pa);
    PIC_LAUNCHED();
}

bool mlp_tc_gemm(const TcGemmOp &g, int E, uint16_t *scratch_a, uint16_t *scratch_b,
                 unsigned int *err, cudaStream_t s) {
    if (g.N < 1 || g.N > NMAX || g.K < 1 || g.K > KMAX || g.M < 1) return false;
    static bool attr[64] = {};   // the shared-memory opt-in, once per device
    const int smem = (int)sizeof(GemmSmem) + 1024;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
        if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return false;
        attr[dev & 63] = true;
    }
    const int Mp = (g.M + TM - 1) / TM * TM, Kp = (g.K + 15) / 16 * 16, Np = (g.N + 15) / 16 * 16;
    // A as an M x K matrix; B as the N x K matrix of its transpose (both K-major)
    k_tc_pack_op<<<dim3(64, E), 256, 0, s>>>(g.A, g.sAz, g.sAm, g.sAk, g.M, g.K, Mp, Kp,
                                             scratch_a, (long long)Mp * Kp);
    PIC_LAUNCHED();
    k_tc_pack_op<<<dim3(64, E), 256, 0, s>>>(g.B, g.sBz, g.sBn, g.sBk, g.N, g.K, Np, Kp,
                                             scratch_b, (long long)Np * Kp);
    PIC_LAUNCHED();
    const TcGemmDev d{scratch_a, scratch_b, (long long)Mp * Kp, (long long)Np * Kp, g.C, g.sCz,
                      g.ldc, g.M, g.N, Kp, Np, g.accumulate, err};
    k_tc_gemm<<<dim3((unsigned)(Mp / TM), (unsigned)E), TM, smem, s>>>(d);
    PIC_LAUNCHED();
    return true;
}

pic_status mlp_tc_forward(const MlpTc &tc, const float *X, float *Y, int64_t n, cudaStream_t s) {
    if (n <= 0) return PIC_OK;
    if (tc.bmember > BIAS_MAX) {
        set_error("pic_mlp_forward: %lld biases per member, the tensor-core path holds %d",
                  tc.bmember, BIAS_MAX);
        return PIC_ERR_ARG;
    }
    const int smem = (int)sizeof(PingSmem) + 1024;
    PIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    PIC_CUDA_TRY(cudaMemsetAsync(tc.err, 0, sizeof(unsigned int), s));
    // grid: members along x, pairs of tiles along y (at most 65535 pairs per launch)
    const long long pairs = (n + NTILE * TM - 1) / (NTILE * TM);
    for (long long p0 = 0; p0 < pairs; p0 += 65535) {
        const long long np_ = std::min<long long>(65535, pairs - p0);
        k_mlp_tc<<<dim3((unsigned)tc.E, (unsigned)np_), NTH, smem, s>>>(tc, X, Y, (long long)n,
                                                                        p0 * NTILE * TM);
        PIC_LAUNCHED();
    }
    PIC_CUDA_TRY(cudaGetLastError());
    unsigned int err = 0;
    PIC_CUDA_TRY(cudaMemcpyAsync(&err, tc.err, sizeof(err), cudaMemcpyDeviceToHost, s));
    PIC_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) {
        set_error("pic_mlp_forward: %u tensor-core waits timed out", err);
        return PIC_ERR_TIMEOUT;
    }
    return PIC_OK;
}

}  // namespace pic
