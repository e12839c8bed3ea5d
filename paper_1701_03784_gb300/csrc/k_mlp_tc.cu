// Surrogate network inference on the 5th-generation tensor cores: BF16 operands in shared
// memory, FP32 accumulation in tensor memory (TMEM).
//
// One CTA of 128 threads takes 128 samples of one ensemble member through every layer:
//  * the activations (128 x K) and the layer's weights (N x K) sit in shared memory in the
//    no-swizzle K-major layout (8 x 8 core matrices of 16-byte rows, K-adjacent core
//    matrices 128 bytes apart, 8-row groups K/8 x 128 bytes apart);
//  * one thread issues tcgen05.mma (kind::f16, M = 128, N = the padded layer width), 16
//    of K at a time, accumulating a 128 x N FP32 tile in TMEM, and commits to an mbarrier;
//  * each warp reads its 32 TMEM lanes (sample rows) with tcgen05.ld, adds the bias,
//    applies the tanh-GELU (hidden layers) and writes the next layer's BF16 operand back
//    into shared memory, or writes the FP32 outputs.
// Every mbarrier wait is bounded (timeout counted, TMEM still freed).
#include <cuda_bf16.h>

#include "pic_internal.h"

namespace pic {

namespace {
constexpr int TM = 128;       // samples per CTA = MMA M
constexpr int NTH = 256;      // 8 warps: two per TMEM lane quadrant, each half the columns
constexpr int KMAX = 256;
constexpr int NMAX = 256;
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1LL << 22;
constexpr float C_GELU = 0.7978845608028654f;   // sqrt(2/pi)

struct TcSmem {
    uint16_t a[TM * KMAX];     // activations, core-matrix layout
    uint16_t w[NMAX * KMAX];   // weights of the current layer, core-matrix layout
    float bias[2][NMAX];       // biases of the current and the next layer
    unsigned long long mbar;   // products of a layer done
    unsigned long long wbar;   // weights and bias of a layer landed
    unsigned int tmem;
};

// element offset of (row r, column k) in a core-matrix tile with kp (padded) columns
__host__ __device__ __forceinline__ int core_off(int r, int k, int kp) {
    return ((r >> 3) * (kp >> 3) * 64) + ((k >> 3) * 64) + ((r & 7) * 8) + (k & 7);
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
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    for (long long k = 0; k < WAIT_LIMIT; k++) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// tanh-GELU with the hardware tanh approximation (relative error about 2^-11, below the
// BF16 rounding of the result)
__device__ __forceinline__ float gelu_approx(float z) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(C_GELU * (z + 0.044715f * z * z * z)));
    return 0.5f * z * (1.f + t);
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
// 8 values as 8 BF16 in one 16-byte word (element 0 lowest)
__device__ __forceinline__ uint4 pack8(const float *v) {
    uint4 q;
    q.x = (unsigned)bf16_bits(v[0]) | ((unsigned)bf16_bits(v[1]) << 16);
    q.y = (unsigned)bf16_bits(v[2]) | ((unsigned)bf16_bits(v[3]) << 16);
    q.z = (unsigned)bf16_bits(v[4]) | ((unsigned)bf16_bits(v[5]) << 16);
    q.w = (unsigned)bf16_bits(v[6]) | ((unsigned)bf16_bits(v[7]) << 16);
    return q;
}
// one thread: fetch layer l's weights (core-matrix layout, np x kp BF16) and bias (np FP32,
// into bias buffer l % 2), completing on wbar
__device__ __forceinline__ void load_layer(const MlpTc &tc, TcSmem &sm, int z, int l) {
    const unsigned wb = (unsigned)(tc.np[l] * tc.kp[l] * 2), bb = (unsigned)(tc.np[l] * 4);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(&sm.wbar)), "r"(wb + bb) : "memory");
    bulk_load(sm.w, tc.w + (long long)z * tc.wmember + tc.woff[l], wb, &sm.wbar);
    bulk_load(sm.bias[l & 1], tc.b + (long long)z * tc.bmember + tc.boff[l], bb, &sm.wbar);
}

__global__ void __launch_bounds__(NTH, 1) k_mlp_tc(MlpTc tc, const float *X, float *Y,
                                                   long long n) {
    extern __shared__ unsigned char raw[];
    const unsigned pad = (1024u - (smem_u32(raw) & 1023u)) & 1023u;
    TcSmem &sm = *reinterpret_cast<TcSmem *>(raw + pad);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.y;
    const long long row0 = (long long)blockIdx.x * TM;
    // epilogue: warp w reads TMEM lane quadrant w % 4 (rows) and half w / 4 of the columns
    const int quad = warp & 3, half = warp >> 2;
    const int erow = quad * 32 + lane;

    if (tid == 0) {
        mbar_init(&sm.mbar, 1);
        mbar_init(&sm.wbar, 1);
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
    if (tid == 0) load_layer(tc, sm, z, 0);
    // layer-0 operand: one sample per thread of the first 128, BF16, zero-padded
    if (tid < TM) {
        const long long row = row0 + tid;
        const int k0 = tc.k[0], kp = tc.kp[0];
        for (int c = 0; c < kp; c += 8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int kk = c + j;
                v[j] = row < n && kk < k0 ? X[row * k0 + kk] : 0.f;
            }
            *reinterpret_cast<uint4 *>(sm.a + core_off(tid, c, kp)) = pack8(v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();

    bool ok = true;
    for (int l = 0; l < tc.L && ok; l++) {
        const int kp = tc.kp[l], np = tc.np[l];
        const bool last = l == tc.L - 1;
        // the layer's weights and bias have landed
        ok = __syncthreads_and(mbar_wait(&sm.wbar, (unsigned)(l & 1)));
        if (!ok) break;
        if (tid == 0) {
            fence_after();
            const unsigned a0 = smem_u32(sm.a), w0 = smem_u32(sm.w);
            const unsigned sbo = (unsigned)kp / 8u * 128u;
            const unsigned id = idesc_bf16(np);
            for (int kk = 0; kk < kp / 16; kk++)
                mma_bf16(tmem, sdesc(a0 + kk * 256u, 128u, sbo), sdesc(w0 + kk * 256u, 128u, sbo),
                         id, kk > 0);
            mma_commit(&sm.mbar);
        }
        ok = __syncthreads_and(mbar_wait(&sm.mbar, (unsigned)(l & 1)));
        if (!ok) break;
        fence_after();
        // the products are done with the weight buffer: fetch the next layer's during the
        // epilogue (its bias goes to the other bias buffer)
        if (tid == 0 && !last) load_layer(tc, sm, z, l + 1);
        const float *bias = sm.bias[l & 1];
        const int chunks = np / 16, c0 = half ? (chunks + 1) / 2 : 0;
        const int c1 = half ? chunks : (chunks + 1) / 2;
        const long long row = row0 + erow;
        for (int ch = c0; ch < c1; ch++) {
            const int c = ch * 16;
            float v[16];
            tmem_ld16(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)c, v);
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] += bias[c + j];
            if (!last) {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = gelu_approx(v[j]);
                *reinterpret_cast<uint4 *>(sm.a + core_off(erow, c, np)) = pack8(v);
                *reinterpret_cast<uint4 *>(sm.a + core_off(erow, c + 8, np)) = pack8(v + 8);
            } else if (row < n) {
                const int nout = tc.n[l];
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (c + j < nout) Y[((long long)z * n + row) * nout + c + j] = v[j];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
    }
    if (!ok) {
        // a wait gave up: count it, give the copies and products in flight one more bounded
        // wait, free TMEM below
        if (tid == 0) {
            atomicAdd(tc.err, 1u);
            mbar_wait(&sm.wbar, 0);
            mbar_wait(&sm.wbar, 1);
            mbar_wait(&sm.mbar, 0);
            mbar_wait(&sm.mbar, 1);
        }
        __syncthreads();
    }
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS) : "memory");
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
        dst[core_off(r, c, kp)] = bf16_bits(r < nn && c < k ? W[(long long)r * k + c] : 0.f);
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
    const int smem = (int)sizeof(TcSmem) + 1024;
    PIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PIC_CUDA_TRY(cudaMemsetAsync(tc.err, 0, sizeof(unsigned int), s));
    dim3 grid((unsigned)((n + TM - 1) / TM), (unsigned)tc.E);
    k_mlp_tc<<<grid, NTH, smem, s>>>(tc, X, Y, (long long)n);
    PIC_LAUNCHED();
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
