// Surrogate network of the batched disk sweep: bfloat16 tensor-core products
// with FP32 accumulation for the forward pass, back-propagation and Adam.
// The contract of each entry point is in include/fargo_mlp.h.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/fargo.h"
#include "../../include/fargo_mlp.h"

namespace mlp {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// Products C[m][n] = sum_k A^[m][k] B^[n][k] with fused epilogues.  A^[m][k]
// is A[m*lda + k], or A[k*lda + m] when TA; B^[n][k] likewise with TB.
// ---------------------------------------------------------------------------
enum { EPI_HIDDEN, EPI_OUT, EPI_STORE, EPI_DA };

struct GemmArgs {
    const bf16 *A, *B;
    int lda, ldb, M, N, K;
    // EPI_HIDDEN: Z = acc + bias (FP32), Ab = bf16(relu(Z))
    // EPI_OUT:    C = (acc + bias) * oscale + oshift (FP32)
    // EPI_STORE:  C = acc (FP32)
    // EPI_DA:     acc masked by Zmask > 0 -> C (FP32) and Ab (bf16)
    float *C;
    bf16 *Ab;
    const float *bias, *Zmask, *oshift, *oscale;
    int ldc;
    int ldab;   // row pitch of Ab (EPI_HIDDEN: the padded activation pitch)
    int *err;   // timeout flag (tcgen05 kernel)
};

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------
// The products run on the fifth-generation tensor cores (tcgen05).  One CTA
// of four warps computes a 128 x 256 tile of C with its FP32 accumulator in
// tensor memory (TMEM: 128 lanes = rows, 256 columns).  K advances in
// 64-deep chunks through two shared-memory stages holding A^ (128 x 64) and
// B^ (256 x 64) in the canonical K-major layout without swizzle: 8 x 8
// "core matrices" of 128 contiguous bytes (8 rows of 16 bytes), K-adjacent
// core matrices 128 bytes apart (leading offset) and 8-row groups 1024
// bytes apart (stride offset).  All threads stage a chunk with plain loads
// (transposing when TA / TB), then one thread issues four
// tcgen05.mma.kind::f16 (K = 16 each, bfloat16 operands, FP32 accumulate)
// and commits them to the stage's mbarrier, which releases the stage two
// chunks later.  The epilogue reads the accumulator row by row with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and applies the fused
// epilogue.  Every wait is bounded; on expiry
// the CTA records the timeout, skips the epilogue and still frees its TMEM.
// ---------------------------------------------------------------------------
namespace tc {

constexpr int TM = 128, TN = 256, TK = 64, NTH = 128;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = 2 * STAGE_BYTES;   // 96 KB: at most two CTAs (512 TMEM columns) per SM
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const unsigned a = su32(bar);
    for (unsigned it = 0; it < kWaitLimit; it++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Shared-memory matrix descriptor: K-major, no swizzle (layout type 0),
// descriptor version 1; lbo = byte distance of K-adjacent core matrices,
// sbo = byte distance of adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo = 128, unsigned sbo = 1024)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Shared-memory matrix descriptor of the K-major 128-byte-swizzle layout:
// rows of 128 bytes, 8-row atoms 1024 bytes apart (stride offset), leading
// offset unused (encoded 1), layout type 2 (128-byte swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(unsigned saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B,
// both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

// byte offset of element (r, k) of a staged chunk
__device__ __forceinline__ unsigned core_off(int r, int k)
{
    return (unsigned)((((r >> 3) * (TK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

template <bool TX>
__device__ __forceinline__ void stage(unsigned char *dst, int rows, const bf16 *X, int ld, int R, int Kd, int r0,
                                      int k0)
{
    const bf16 zero = __float2bfloat16(0.0f);
    for (int idx = threadIdx.x; idx < rows * TK; idx += NTH) {
        int r, k;
        if (TX) {
            r = idx % rows;
            k = idx / rows;
        } else {
            r = idx / TK;
            k = idx % TK;
        }
        const int gr = r0 + r, gk = k0 + k;
        bf16 v = zero;
        if (gr < R && gk < Kd) v = TX ? X[(size_t)gk * ld + gr] : X[(size_t)gr * ld + gk];
        *reinterpret_cast<bf16 *>(dst + core_off(r, k)) = v;
    }
}

// Epilogue of a 128 x TN accumulator tile.  Warp w owns TMEM lanes
// 32w..32w+31 (rows m0+32w..); per 32-column slice it reads its 32 x 32
// block with two tcgen05.ld, parks it in shared memory (row pitch 33 floats:
// conflict-free both ways) and then writes it row by row, lane = column, so
// every store instruction covers one contiguous row segment.  `tile` is the
// warp's 32 x 33 float scratch (the operand stages are free by then).
// EPI_HIDDEN with C == nullptr stores only the activations (inference).
template <int EPI>
__device__ __forceinline__ void epilogue(const GemmArgs &g, uint32_t tmem, int m0, int n0, float *tile)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rbase = m0 + warp * 32;
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 32) {
        if (n0 + c0 >= g.N || rbase >= g.M) break;   // warp-uniform
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15}, [%16];"
            : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr + 16u));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int u = 0; u < 32; u++) tile[lane * 33 + u] = __uint_as_float(r[u]);
        __syncwarp();
        const int col = n0 + c0 + lane;
        const bool cok = col < g.N;
        float b = 0.0f, sc = 1.0f, sh = 0.0f;
        if (cok && (EPI == EPI_HIDDEN || EPI == EPI_OUT)) b = g.bias[col];
        if (cok && EPI == EPI_OUT) {
            sc = g.oscale[col];
            sh = g.oshift[col];
        }
        const int nr = min(32, g.M - rbase);
#pragma unroll 4
        for (int rr = 0; rr < nr; rr++) {
            float v = tile[rr * 33 + lane];
            if (!cok) continue;
            const int row = rbase + rr;
            const size_t o = (size_t)row * g.ldc + col;
            if (EPI == EPI_HIDDEN) {
                v += b;
                if (g.C) g.C[o] = v;
                g.Ab[(size_t)row * g.ldab + col] = __float2bfloat16_rn(v > 0.0f ? v : 0.0f);
            } else if (EPI == EPI_OUT) {
                g.C[o] = (v + b) * sc + sh;
            } else if (EPI == EPI_STORE) {
                g.C[o] = v;
            } else {
                v = g.Zmask[o] > 0.0f ? v : 0.0f;
                g.C[o] = v;
                g.Ab[o] = __float2bfloat16_rn(v);
            }
        }
        __syncwarp();
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(NTH, 1) k_gemm_tc(GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"((unsigned)TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int nk = (g.K + TK - 1) / TK;
    bool ok = true;
    for (int kc = 0; kc < nk && ok; kc++) {
        const int st = kc & 1;
        unsigned char *sa = smem + st * STAGE_BYTES, *sb = sa + A_BYTES;
        // the MMAs of chunk kc-2 read this stage: wait for their commit
        if (kc >= 2) ok = mbar_wait(&bar[st], ((kc - 2) >> 1) & 1);
        if (!__syncthreads_and(ok)) break;
        stage<TA>(sa, TM, g.A, g.lda, g.M, g.K, m0, kc * TK);
        stage<TB>(sb, TN, g.B, g.ldb, g.N, g.K, n0, kc * TK);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = su32(sa), b0 = su32(sb);
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++) {
                const uint64_t ad = smem_desc(a0 + kk * 256), bd = smem_desc(b0 + kk * 256);
                const unsigned acc = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar[st]))
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && nk > 0) ok = mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        epilogue<EPI>(g, tmem, m0, n0, reinterpret_cast<float *>(smem) + warp * 32 * 33);
    } else if (threadIdx.x == 0) {
        atomicOr(g.err, 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)TN)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Forward products with TMA staging.  Both operands are K-contiguous (the
// activations [rows][K] and the weights [N][K], rows 16-byte aligned), so
// thread 0 stages a 64-deep chunk with one 2D tensor-map load per operand:
// box 64 K x 128 rows for A, 64 x 256 for B, 128-byte swizzle.  A row of the
// box is 128 bytes (the chunk's 64 K values), eight rows form a 1024-byte
// swizzle atom, so the MMA descriptors use the 128-byte-swizzle K-major
// layout with a stride offset of 1024 bytes, and the K = 16 step inside the
// chunk advances the start address by 32 bytes (the swizzle is applied to
// the absolute shared address, hence the 1024-byte aligned stages).
// Out-of-range rows and K columns read as zero.  Thread 0 prefetches chunk
// kc+1 while the tensor cores work on chunk kc; every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(NTH, 1) k_gemm_tma(const __grid_constant__ CUtensorMap ma,
                                                    const __grid_constant__ CUtensorMap mb, GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2], done[2];
    // swizzled stages start on a 1024-byte boundary (the launch adds 1 KB)
    unsigned char *sm = smem + ((1024u - (su32(smem) & 1023u)) & 1023u);
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"((unsigned)TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int nk = (g.K + TK - 1) / TK;
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&ma) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mb) : "memory");
        auto issue = [&](int kc) {
            const int st = kc & 1;
            unsigned char *sa = sm + st * STAGE_BYTES, *sb = sa + A_BYTES;
            mbar_expect_tx(&full[st], (unsigned)STAGE_BYTES);
            tma_load_2d(sa, &ma, kc * TK, m0, &full[st]);
            tma_load_2d(sb, &mb, kc * TK, n0, &full[st]);
        };
        bool ok = true;
        int issued = 0;   // chunks whose copies were issued
        if (nk > 0) {
            issue(0);
            issued = 1;
        }
        for (int kc = 0; kc < nk && ok; kc++) {
            const int st = kc & 1;
            if (kc + 1 < nk) {
                // chunk kc-1 used the other stage: its MMAs must be done
                if (kc >= 1) ok = mbar_wait(&done[(kc + 1) & 1], ((kc - 1) >> 1) & 1);
                if (!ok) break;
                issue(kc + 1);
                issued = kc + 2;
            }
            ok = mbar_wait(&full[st], (kc >> 1) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = su32(sm + st * STAGE_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++) {
                const uint64_t ad = smem_desc_sw128(a0 + kk * 32);
                const uint64_t bd = smem_desc_sw128(b0 + kk * 32);
                const unsigned acc = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&done[st]))
                         : "memory");
        }
        if (ok && nk > 0) ok = mbar_wait(&done[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
        if (!ok) {
            // let the copies in flight land before the CTA can leave
            for (int kc = 0; kc < issued; kc++) mbar_wait(&full[kc & 1], (kc >> 1) & 1);
        }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_ok) {
        epilogue<EPI>(g, tmem, m0, n0, reinterpret_cast<float *>(sm) + warp * 32 * 33);
    } else if (threadIdx.x == 0) {
        atomicOr(g.err, 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)TN)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Whole-network inference in one kernel.  A CTA owns 128 samples and keeps
// them on chip through every layer: their activations in shared memory
// (bfloat16, the 128-byte-swizzle K-major layout the MMA reads, up to five
// 64-deep chunks), the layer's accumulator in tensor memory.  Only the
// weights stream in, by TMA, in 32 KB chunks (64 K x 256 rows) through four
// stages that run ahead across layer boundaries, so the next layer's weights
// arrive while the current layer's epilogue runs.  Per layer:
//  - thread 0 issues the layer's MMAs chunk by chunk (each chunk as soon as
//    its weights land; the stage of the previous chunk is refilled once its
//    MMAs completed) and commits the layer to an mbarrier;
//  - all eight warps drain the accumulator (warp w: TMEM lanes 32 (w % 4)..,
//    columns 128 (w / 4)..): bias and ReLU, rounded to bfloat16 and written
//    back into the activation chunks, or, after the last layer, the output
//    map and row-coalesced FP32 stores through shared memory;
//  - a proxy fence and a barrier hand the new activations to the next
//    layer's MMAs.
// The input map and the rounding to bfloat16 happen here too, from the FP32
// input rows.  The arithmetic is that of the layer-by-layer products: the
// same operands, chunking and MMA shapes.  Networks with an input of at most
// 320 features, layers of at most 256 and at most 8 layers qualify.
// ---------------------------------------------------------------------------
constexpr int F_THREADS = 256, F_MAXL = 8, F_ACT = 5, F_STAGES = 4;
constexpr int F_CHUNK_A = 128 * 128, F_CHUNK_W = 256 * 128;
constexpr int F_SMEM = F_ACT * F_CHUNK_A + F_STAGES * F_CHUNK_W + F_MAXL * 256 * 4 + 1024;

struct FusedArgs {
    const float *x;
    float *y;
    const float *shift, *scale, *oshift, *oscale;
    const float *bias[F_MAXL];
    int dims[F_MAXL + 1];
    int L, M;
    int *err;
};
struct FusedMaps {
    CUtensorMap w[F_MAXL];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
// byte offset of the 16-byte unit u (8 values along K) of row r in a
// 128-byte-swizzled 128-row chunk
__device__ __forceinline__ unsigned sw128_off(int r, int u) { return (unsigned)(r * 128 + ((u ^ (r & 7)) << 4)); }

__global__ void __launch_bounds__(F_THREADS, 1) k_mlp_fused(const __grid_constant__ FusedMaps fm,
                                                          const __grid_constant__ FusedArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t wfull[F_STAGES], wempty[F_STAGES], accb;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    unsigned char *sm = smem + ((1024u - (su32(smem) & 1023u)) & 1023u);
    unsigned char *act = sm;
    unsigned char *wst = sm + F_ACT * F_CHUNK_A;
    float *sbias = reinterpret_cast<float *>(wst + F_STAGES * F_CHUNK_W);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, L = a.L;
    int total = 0;
    for (int l = 0; l < L; l++) total += (a.dims[l] + 63) / 64;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < F_STAGES; q++) {
            mbar_init(&wfull[q], 1);
            mbar_init(&wempty[q], 1);
        }
        mbar_init(&accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    for (int i = tid; i < L * 256; i += F_THREADS) {
        const int l = i >> 8, c = i & 255;
        sbias[i] = c < a.dims[l + 1] ? a.bias[l][c] : 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // thread 0: weight chunk gg of the whole network into stage gg % 4
    int issued = 0;
    auto issue_w = [&](int gg) {
        int l = 0, c = gg;
        while (c >= (a.dims[l] + 63) / 64) {
            c -= (a.dims[l] + 63) / 64;
            l++;
        }
        const int st = gg & (F_STAGES - 1);
        mbar_expect_tx(&wfull[st], (unsigned)F_CHUNK_W);
        tma_load_2d(wst + st * F_CHUNK_W, &fm.w[l], c * 64, 0, &wfull[st]);
        issued = gg + 1;
    };
    if (tid == 0) {
        for (int l = 0; l < L; l++) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&fm.w[l]) : "memory");
        for (int gg = 0; gg < F_STAGES && gg < total; gg++) issue_w(gg);
    }
    // the input rows: (x - shift) * scale rounded to bfloat16, zero beyond the
    // batch and the features.  Thread t owns the 8-feature unit t % units of
    // every (F_THREADS / units)-th row, with that unit's shift and scale in
    // registers; the loads of eight rows are issued before any is stored.
    {
        const int K0 = a.dims[0], units = ((K0 + 63) / 64) * 8;
        const int rstep = F_THREADS / units, u = tid % units, k0 = u * 8;
        if (tid < units * rstep) {
            float sh[8], sc[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int k = k0 + e;
                sh[e] = k < K0 ? a.shift[k] : 0.0f;
                sc[e] = k < K0 ? a.scale[k] : 0.0f;
            }
            constexpr int RB = 8;
            for (int rb = tid / units; rb < 128; rb += RB * rstep) {
                float v[RB][8];
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    const int r = rb + j * rstep, row = m0 + r;
#pragma unroll
                    for (int e = 0; e < 8; e++)
                        v[j][e] = r < 128 && row < a.M && k0 + e < K0 ? a.x[(size_t)row * K0 + k0 + e] : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    const int r = rb + j * rstep, row = m0 + r;
                    if (r >= 128) break;
                    float f[8];
#pragma unroll
                    for (int e = 0; e < 8; e++) f[e] = row < a.M && k0 + e < K0 ? (v[j][e] - sh[e]) * sc[e] : 0.0f;
                    const unsigned off = (unsigned)((u >> 3) * F_CHUNK_A) + sw128_off(r, u & 7);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(su32(act + off)),
                                 "r"(pack_bf16(f[0], f[1])), "r"(pack_bf16(f[2], f[3])),
                                 "r"(pack_bf16(f[4], f[5])), "r"(pack_bf16(f[6], f[7]))
                                 : "memory");
                }
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    int g = 0;
    const int q4 = warp & 3, h = warp >> 2;
    const int r = q4 * 32 + lane;   // the thread's accumulator row
    for (int l = 0; l < L; l++) {
        const int nk = (a.dims[l] + 63) / 64;
        if (tid == 0) {
            bool ok = s_fail == 0;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int kc = 0; kc < nk && ok; kc++, g++) {
                const int st = g & (F_STAGES - 1);
                ok = mbar_wait(&wfull[st], (g >> 2) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned a0 = su32(act + kc * F_CHUNK_A), b0 = su32(wst + st * F_CHUNK_W);
#pragma unroll
                for (int kk = 0; kk < 4; kk++) {
                    const uint64_t ad = smem_desc_sw128(a0 + kk * 32), bd = smem_desc_sw128(b0 + kk * 32);
                    const unsigned acc = (kc > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&wempty[st]))
                             : "memory");
                // refill the previous chunk's stage once its MMAs are done
                if (g >= 1 && g + F_STAGES - 1 < total) {
                    const int ps = (g - 1) & (F_STAGES - 1);
                    ok = mbar_wait(&wempty[ps], ((g - 1) >> 2) & 1);
                    if (!ok) break;
                    issue_w(g + F_STAGES - 1);
                }
            }
            if (ok)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&accb))
                             : "memory");
            else
                s_fail = 1;
        }
        // every thread waits for the layer's accumulator (bounded)
        const bool got = mbar_wait(&accb, l & 1);
        if (!got) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float *bl = sbias + l * 256;
        const bool last = l == L - 1;
        float *tile = reinterpret_cast<float *>(wst) + warp * 32 * 33;
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {
            const int cb = h * 128 + c0;
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)cb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                  "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr + 16u));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!last) {
                // bias, ReLU, bfloat16: four 16-byte units of the next layer's input
#pragma unroll
                for (int uu = 0; uu < 4; uu++) {
                    float f[8];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const float z = __uint_as_float(v[uu * 8 + e]) + bl[cb + uu * 8 + e];
                        f[e] = z > 0.0f ? z : 0.0f;
                    }
                    const int col = cb + uu * 8;
                    const unsigned off = (unsigned)((col >> 6) * F_CHUNK_A) + sw128_off(r, (col & 63) >> 3);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(su32(act + off)),
                                 "r"(pack_bf16(f[0], f[1])), "r"(pack_bf16(f[2], f[3])),
                                 "r"(pack_bf16(f[4], f[5])), "r"(pack_bf16(f[6], f[7]))
                                 : "memory");
                }
            } else {
                // output map, stored row by row (lane = column) through the
                // warp's 32 x 33 scratch in the now idle weight stages
#pragma unroll
                for (int e = 0; e < 32; e++) tile[lane * 33 + e] = __uint_as_float(v[e]);
                __syncwarp();
                const int col = cb + lane, N = a.dims[L];
                if (col < N) {
                    const float b = bl[col], sc = a.oscale[col], sh = a.oshift[col];
                    for (int rr = 0; rr < 32; rr++) {
                        const int row = m0 + q4 * 32 + rr;
                        if (row < a.M) a.y[(size_t)row * N + col] = (tile[rr * 33 + lane] + b) * sc + sh;
                    }
                }
                __syncwarp();
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) {
            atomicOr(a.err, 4);
            // let the weight copies in flight land, and the MMAs finish
            for (int gg = g; gg < issued; gg++) mbar_wait(&wfull[gg & (F_STAGES - 1)], (gg >> 2) & 1);
            if (g > 0) mbar_wait(&wempty[(g - 1) & (F_STAGES - 1)], ((g - 1) >> 2) & 1);
        }
        __syncthreads();
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
    }
}

}  // namespace tc

template <bool TA, bool TB, int EPI>
static void gemm(const GemmArgs &g, cudaStream_t s)
{
    const dim3 grid((g.N + tc::TN - 1) / tc::TN, (g.M + tc::TM - 1) / tc::TM);
    tc::k_gemm_tc<TA, TB, EPI><<<grid, tc::NTH, tc::SMEM_BYTES, s>>>(g);
}

template <bool TA, bool TB, int EPI>
static cudaError_t gemm_attr()
{
    return cudaFuncSetAttribute(tc::k_gemm_tc<TA, TB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES);
}

template <int EPI>
static void gemm_tma(const CUtensorMap &ma, const CUtensorMap &mb, const GemmArgs &g, cudaStream_t s)
{
    const dim3 grid((g.N + tc::TN - 1) / tc::TN, (g.M + tc::TM - 1) / tc::TM);
    tc::k_gemm_tma<EPI><<<grid, tc::NTH, tc::SMEM_BYTES + 1024, s>>>(ma, mb, g);
}

template <int EPI>
static cudaError_t gemm_tma_attr()
{
    return cudaFuncSetAttribute(tc::k_gemm_tma<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES + 1024);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2D map of a bfloat16 matrix [rows][cols] with row pitch `ld` values (a
// multiple of 8), box of 64 columns (128 bytes) by box_rows rows, 128-byte
// swizzle, zero fill outside.
static bool encode_bf16(CUtensorMap *map, const bf16 *base, int cols, int rows, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)tc::TK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Where each layer's weights sit in the flat parameter vector, and their
// padded bfloat16 copies (row pitch a multiple of 8) for the tensor maps.
struct LayerTab {
    int L;
    unsigned long long woff[16];
    int K[16], N[16], ldp[16];
    bf16 *wpad[16];
};

__device__ __forceinline__ void pack_weight(const LayerTab &lt, size_t i, bf16 v)
{
    for (int l = 0; l < lt.L; l++) {
        const size_t rel = i - (size_t)lt.woff[l];
        if (i >= (size_t)lt.woff[l] && rel < (size_t)lt.K[l] * lt.N[l]) {
            const size_t n = rel / lt.K[l], k = rel - n * lt.K[l];
            lt.wpad[l][n * lt.ldp[l] + k] = v;
            return;
        }
    }
}

// x' = bf16((x - shift) * scale), rows of `cols` values written with pitch
// ld (the padding columns hold zeros)
__global__ void k_input(const float *x, int rows, int cols, int ld, const float *shift, const float *scale,
                        bf16 *out)
{
    const int n = rows * ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i / ld, c = i - r * ld;
        out[i] = c < cols ? __float2bfloat16_rn((x[(size_t)r * cols + c] - shift[c]) * scale[c])
                          : __float2bfloat16(0.0f);
    }
}

// Mean-squared error of y = z * oscale + oshift and its gradient with respect
// to z, 2 (y - t) oscale / count; one block with a fixed-shape reduction
// (deterministic).
__global__ void __launch_bounds__(1024) k_mse(const float *y, const float *t, int count, int cols,
                                              const float *oscale, float *dz, bf16 *dzb, float *loss)
{
    __shared__ float red[32];
    const float s2 = 2.0f / (float)count;
    float acc = 0.0f;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const float d = y[i] - t[i];
        acc += d * d;
        const float gz = s2 * d * oscale[i % cols];
        dz[i] = gz;
        dzb[i] = __float2bfloat16_rn(gz);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) *loss = v / (float)count;
    }
}

// Bias gradients: column sums of dz [rows][cols], one thread per column.
__global__ void k_colsum(const float *dz, int rows, int cols, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; r++) s += dz[(size_t)r * cols + c];
    db[c] = s;
}

struct AdamHyper {
    float lr, b1, b2, eps;
    int t;
};

__global__ void k_adam_tick(AdamHyper *h) { h->t += 1; }

// Adam on the flat parameter vector; bfloat16 copies (flat and padded) re-rounded.
__global__ void k_adam(float *w, float *m, float *v, const float *g, bf16 *wb, size_t n, const AdamHyper *h,
                       LayerTab lt)
{
    const float lr = h->lr, b1 = h->b1, b2 = h->b2, eps = h->eps;
    const float t = (float)h->t;
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        const bf16 b = __float2bfloat16_rn(wi);
        wb[i] = b;
        pack_weight(lt, i, b);
    }
}

__global__ void k_round(const float *w, bf16 *wb, size_t n, LayerTab lt)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const bf16 b = __float2bfloat16_rn(w[i]);
        wb[i] = b;
        pack_weight(lt, i, b);
    }
}

// One block per sample: ensemble mean and relative spread.
__global__ void __launch_bounds__(256) k_ensemble(const float *ys, int k, int batch, int n, float *mean,
                                                   float *spread)
{
    __shared__ float r1[8], r2[8];
    const int b = blockIdx.x;
    float sv = 0.0f, sm = 0.0f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float mu = 0.0f;
        for (int e = 0; e < k; e++) mu += ys[((size_t)e * batch + b) * n + j];
        mu /= (float)k;
        float var = 0.0f;
        for (int e = 0; e < k; e++) {
            const float d = ys[((size_t)e * batch + b) * n + j] - mu;
            var += d * d;
        }
        var /= (float)(k - 1);
        mean[(size_t)b * n + j] = mu;
        sv += var;
        sm += mu * mu;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = sv;
        r2[threadIdx.x >> 5] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.0f, c = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a += r1[w];
            c += r2[w];
        }
        spread[b] = c > 0.0f ? sqrtf(a / c) : 0.0f;
    }
}

}  // namespace mlp

using namespace mlp;

struct fargo_mlp {
    std::vector<int> dims;
    int L = 0, max_batch = 0;
    size_t np = 0;
    std::vector<size_t> woff, boff;   // offsets of W_l and b_l in the parameter vector
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 master, moments, gradients
    bf16 *wb = nullptr;                                            // bfloat16 copy (same layout)
    float *shift = nullptr, *scale = nullptr;      // input map
    float *oshift = nullptr, *oscale = nullptr;    // output map
    bf16 *xb = nullptr;                                            // bfloat16 input, pitch ldp[0]
    std::vector<int> ldp;                                          // padded widths (multiples of 8)
    std::vector<bf16 *> wpad;                                      // padded bfloat16 weights per layer
    std::vector<CUtensorMap> mapA, mapB;                           // forward operands per layer
    bool fused = false;                                            // inference in one kernel (k_mlp_fused)
    tc::FusedMaps fmaps{};                                         // its weight maps
    LayerTab lt{};
    std::vector<float *> Z;                                        // hidden pre-activations (FP32)
    std::vector<bf16 *> Ab;                                        // hidden activations (bf16, pitch ldp[l+1])
    float *y = nullptr;                                            // output of the last forward
    float *dz[2] = {nullptr, nullptr};
    bf16 *dzb[2] = {nullptr, nullptr};
    AdamHyper *hyper = nullptr;
    int *err = nullptr;                                            // timeout flag of the products
    std::vector<void *> allocs;
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[4] = {nullptr, nullptr, nullptr, nullptr};
    int gbatch = 0;
};

#define MK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            fprintf(stderr, "fargo_mlp: %s failed: %s\n", #call, cudaGetErrorString(e_));     \
            return e_ == cudaErrorMemoryAllocation ? FARGO_ERR_OOM : FARGO_ERR_CUDA;           \
        }                                                                                     \
    } while (0)

template <typename P>
static int nalloc(fargo_mlp *n, P **p, size_t count)
{
    void *q = nullptr;
    MK(cudaMalloc(&q, (count ? count : 1) * sizeof(P)));
    n->allocs.push_back(q);
    MK(cudaMemsetAsync(q, 0, (count ? count : 1) * sizeof(P), n->stream));
    *p = (P *)q;
    return FARGO_OK;
}

static unsigned blocks_for(size_t n, int bs)
{
    size_t b = (n + bs - 1) / bs;
    return (unsigned)(b > 4096 ? 4096 : (b ? b : 1));
}

extern "C" int fargo_mlp_create(fargo_mlp **out, const int *dims, int nlayers, int max_batch, void *stream)
{
    if (!out || !dims || nlayers < 1 || nlayers > 16 || max_batch < 1) return FARGO_ERR_BADARG;
    *out = nullptr;
    for (int l = 0; l <= nlayers; l++)
        if (dims[l] < 1 || dims[l] > 4096) return FARGO_ERR_BADARG;
    fargo_mlp *n = new fargo_mlp();
    n->dims.assign(dims, dims + nlayers + 1);
    n->L = nlayers;
    n->max_batch = max_batch;
    for (int l = 0; l < nlayers; l++) {
        n->woff.push_back(n->np);
        n->np += (size_t)dims[l] * dims[l + 1];
        n->boff.push_back(n->np);
        n->np += dims[l + 1];
    }
    int rc = FARGO_OK;
    if (stream) {
        n->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) == cudaSuccess) {
        n->own_stream = true;
    } else {
        delete n;
        return FARGO_ERR_CUDA;
    }
    const size_t B = (size_t)max_batch;
    int wmax = 0;
    for (int d : n->dims) wmax = d > wmax ? d : wmax;
    if (!rc) rc = nalloc(n, &n->w, n->np);
    if (!rc) rc = nalloc(n, &n->m, n->np);
    if (!rc) rc = nalloc(n, &n->v, n->np);
    if (!rc) rc = nalloc(n, &n->g, n->np);
    if (!rc) rc = nalloc(n, &n->wb, n->np);
    if (!rc) rc = nalloc(n, &n->shift, dims[0]);
    if (!rc) rc = nalloc(n, &n->scale, dims[0]);
    if (!rc) rc = nalloc(n, &n->oshift, dims[nlayers]);
    if (!rc) rc = nalloc(n, &n->oscale, dims[nlayers]);
    for (int l = 0; l <= nlayers; l++) n->ldp.push_back((dims[l] + 7) / 8 * 8);
    if (!rc) rc = nalloc(n, &n->xb, B * n->ldp[0]);
    for (int l = 0; l < nlayers - 1 && !rc; l++) {
        float *z = nullptr;
        bf16 *a = nullptr;
        rc = nalloc(n, &z, B * dims[l + 1]);
        if (!rc) rc = nalloc(n, &a, B * n->ldp[l + 1]);
        n->Z.push_back(z);
        n->Ab.push_back(a);
    }
    n->lt.L = nlayers;
    for (int l = 0; l < nlayers && !rc; l++) {
        bf16 *wp = nullptr;
        rc = nalloc(n, &wp, (size_t)dims[l + 1] * n->ldp[l]);
        n->wpad.push_back(wp);
        n->lt.woff[l] = n->woff[l];
        n->lt.K[l] = dims[l];
        n->lt.N[l] = dims[l + 1];
        n->lt.ldp[l] = n->ldp[l];
        n->lt.wpad[l] = wp;
    }
    n->mapA.resize(nlayers);
    n->mapB.resize(nlayers);
    for (int l = 0; l < nlayers && !rc; l++) {
        const bf16 *ain = l == 0 ? n->xb : n->Ab[l - 1];
        if (!encode_bf16(&n->mapA[l], ain, dims[l], max_batch, n->ldp[l], tc::TM) ||
            !encode_bf16(&n->mapB[l], n->wpad[l], dims[l], dims[l + 1], n->ldp[l], tc::TN))
            rc = FARGO_ERR_CUDA;
    }
    n->fused = nlayers <= tc::F_MAXL && dims[0] <= 64 * tc::F_ACT;
    for (int l = 1; l <= nlayers; l++) n->fused = n->fused && dims[l] <= 256;
    if (n->fused && !rc) {
        for (int l = 0; l < nlayers; l++) n->fmaps.w[l] = n->mapB[l];
        if (cudaFuncSetAttribute(tc::k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::F_SMEM) !=
            cudaSuccess)
            rc = FARGO_ERR_CUDA;
    }
    if (!rc) rc = nalloc(n, &n->y, B * dims[nlayers]);
    for (int q = 0; q < 2 && !rc; q++) {
        rc = nalloc(n, &n->dz[q], B * wmax);
        if (!rc) rc = nalloc(n, &n->dzb[q], B * wmax);
    }
    if (!rc) rc = nalloc(n, &n->hyper, 1);
    if (!rc) rc = nalloc(n, &n->err, 1);
    if (!rc && (gemm_tma_attr<EPI_HIDDEN>() != cudaSuccess || gemm_tma_attr<EPI_OUT>() != cudaSuccess ||
                gemm_attr<true, true, EPI_STORE>() != cudaSuccess || gemm_attr<false, true, EPI_DA>() != cudaSuccess))
        rc = FARGO_ERR_CUDA;
    if (!rc) {
        std::vector<float> ones(wmax, 1.0f);
        AdamHyper h{1e-3f, 0.9f, 0.999f, 1e-8f, 0};
        if (cudaMemcpyAsync(n->scale, ones.data(), sizeof(float) * dims[0], cudaMemcpyHostToDevice, n->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(n->oscale, ones.data(), sizeof(float) * dims[nlayers], cudaMemcpyHostToDevice,
                            n->stream) != cudaSuccess ||
            cudaMemcpyAsync(n->hyper, &h, sizeof(h), cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
            cudaStreamSynchronize(n->stream) != cudaSuccess)
            rc = FARGO_ERR_CUDA;
    }
    if (rc) {
        fargo_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return FARGO_OK;
}

extern "C" void fargo_mlp_destroy(fargo_mlp *n)
{
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    if (n->gexec) cudaGraphExecDestroy(n->gexec);
    for (void *p : n->allocs) cudaFree(p);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
}

extern "C" size_t fargo_mlp_num_params(const fargo_mlp *n) { return n ? n->np : 0; }

extern "C" int fargo_mlp_set_params(fargo_mlp *n, const float *host, size_t count)
{
    if (!n || !host) return FARGO_ERR_BADARG;
    if (count != n->np) return FARGO_ERR_SIZE;
    MK(cudaMemcpyAsync(n->w, host, n->np * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    MK(cudaMemsetAsync(n->m, 0, n->np * sizeof(float), n->stream));
    MK(cudaMemsetAsync(n->v, 0, n->np * sizeof(float), n->stream));
    k_round<<<blocks_for(n->np, 256), 256, 0, n->stream>>>(n->w, n->wb, n->np, n->lt);
    MK(cudaGetLastError());
    const int zero = 0;
    MK(cudaMemcpyAsync(&n->hyper->t, &zero, sizeof(int), cudaMemcpyHostToDevice, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return FARGO_OK;
}

static int copy_out(fargo_mlp *n, const float *src, float *host, size_t count)
{
    if (!n || !host) return FARGO_ERR_BADARG;
    if (count != n->np) return FARGO_ERR_SIZE;
    MK(cudaMemcpyAsync(host, src, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return FARGO_OK;
}

extern "C" int fargo_mlp_get_params(fargo_mlp *n, float *host, size_t count)
{
    return n ? copy_out(n, n->w, host, count) : FARGO_ERR_BADARG;
}

extern "C" int fargo_mlp_get_grads(fargo_mlp *n, float *host, size_t count)
{
    return n ? copy_out(n, n->g, host, count) : FARGO_ERR_BADARG;
}

extern "C" int fargo_mlp_set_input_map(fargo_mlp *n, const float *shift, const float *scale)
{
    if (!n || !shift || !scale) return FARGO_ERR_BADARG;
    MK(cudaMemcpyAsync(n->shift, shift, sizeof(float) * n->dims[0], cudaMemcpyHostToDevice, n->stream));
    MK(cudaMemcpyAsync(n->scale, scale, sizeof(float) * n->dims[0], cudaMemcpyHostToDevice, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return FARGO_OK;
}

extern "C" int fargo_mlp_set_output_map(fargo_mlp *n, const float *shift, const float *scale)
{
    if (!n || !shift || !scale) return FARGO_ERR_BADARG;
    const int m = n->dims[n->L];
    MK(cudaMemcpyAsync(n->oshift, shift, sizeof(float) * m, cudaMemcpyHostToDevice, n->stream));
    MK(cudaMemcpyAsync(n->oscale, scale, sizeof(float) * m, cudaMemcpyHostToDevice, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return FARGO_OK;
}

extern "C" int fargo_mlp_set_optimizer(fargo_mlp *n, float lr, float b1, float b2, float eps)
{
    if (!n || !(lr > 0.0f) || !(b1 >= 0.0f && b1 < 1.0f) || !(b2 >= 0.0f && b2 < 1.0f) || !(eps >= 0.0f))
        return FARGO_ERR_BADARG;
    AdamHyper h;
    MK(cudaMemcpyAsync(&h, n->hyper, sizeof(h), cudaMemcpyDeviceToHost, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    h.lr = lr;
    h.b1 = b1;
    h.b2 = b2;
    h.eps = eps;
    MK(cudaMemcpyAsync(n->hyper, &h, sizeof(h), cudaMemcpyHostToDevice, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return FARGO_OK;
}

// Forward pass into n->y (hidden pre-activations and activations kept).
// keep_z: store the FP32 pre-activations that back-propagation masks with
// (inference skips them)
static int forward(fargo_mlp *n, const float *x, int batch, bool keep_z)
{
    cudaStream_t s = n->stream;
    const int K0 = n->dims[0];
    k_input<<<blocks_for((size_t)batch * n->ldp[0], 256), 256, 0, s>>>(x, batch, K0, n->ldp[0], n->shift, n->scale,
                                                                      n->xb);
    for (int l = 0; l < n->L; l++) {
        GemmArgs g{};
        g.err = n->err;
        g.M = batch;
        g.N = n->dims[l + 1];
        g.K = n->dims[l];
        g.bias = n->w + n->boff[l];
        g.ldc = g.N;
        if (l < n->L - 1) {
            g.C = keep_z ? n->Z[l] : nullptr;
            g.Ab = n->Ab[l];
            g.ldab = n->ldp[l + 1];
            gemm_tma<EPI_HIDDEN>(n->mapA[l], n->mapB[l], g, s);
        } else {
            g.C = n->y;
            g.oshift = n->oshift;
            g.oscale = n->oscale;
            gemm_tma<EPI_OUT>(n->mapA[l], n->mapB[l], g, s);
        }
    }
    MK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_mlp_forward(fargo_mlp *n, const float *x, int batch, float *y)
{
    if (!n || !x || !y || batch < 1) return FARGO_ERR_BADARG;
    if (batch > n->max_batch) return FARGO_ERR_SIZE;
    if (n->fused) {
        tc::FusedArgs fa{};
        fa.x = x;
        fa.y = y;
        fa.shift = n->shift;
        fa.scale = n->scale;
        fa.oshift = n->oshift;
        fa.oscale = n->oscale;
        for (int l = 0; l < n->L; l++) fa.bias[l] = n->w + n->boff[l];
        for (int l = 0; l <= n->L; l++) fa.dims[l] = n->dims[l];
        fa.L = n->L;
        fa.M = batch;
        fa.err = n->err;
        tc::k_mlp_fused<<<(batch + 127) / 128, tc::F_THREADS, tc::F_SMEM, n->stream>>>(n->fmaps, fa);
        MK(cudaGetLastError());
        return FARGO_OK;
    }
    int rc = forward(n, x, batch, false);
    if (rc) return rc;
    MK(cudaMemcpyAsync(y, n->y, sizeof(float) * batch * n->dims[n->L], cudaMemcpyDeviceToDevice, n->stream));
    return FARGO_OK;
}

static int backward(fargo_mlp *n, const float *x, const float *t, int batch, float *loss)
{
    int rc = forward(n, x, batch, true);
    if (rc) return rc;
    cudaStream_t s = n->stream;
    const int L = n->L;
    int cur = 0;
    k_mse<<<1, 1024, 0, s>>>(n->y, t, batch * n->dims[L], n->dims[L], n->oscale, n->dz[cur], n->dzb[cur], loss);
    for (int l = L - 1; l >= 0; l--) {
        const int No = n->dims[l + 1], Ki = n->dims[l];
        const bf16 *Ain = l == 0 ? n->xb : n->Ab[l - 1];
        // dW_l[o][i] = sum_b dZ[b][o] A[b][i]
        GemmArgs gw{};
        gw.err = n->err;
        gw.A = n->dzb[cur];
        gw.lda = No;
        gw.B = Ain;
        gw.ldb = n->ldp[l];
        gw.M = No;
        gw.N = Ki;
        gw.K = batch;
        gw.C = n->g + n->woff[l];
        gw.ldc = Ki;
        gemm<true, true, EPI_STORE>(gw, s);
        k_colsum<<<(No + 255) / 256, 256, 0, s>>>(n->dz[cur], batch, No, n->g + n->boff[l]);
        if (l > 0) {
            // dZ_{l-1}[b][i] = (Z_{l-1}[b][i] > 0) sum_o dZ[b][o] W_l[o][i]
            GemmArgs ga{};
            ga.err = n->err;
            ga.A = n->dzb[cur];
            ga.lda = No;
            ga.B = n->wb + n->woff[l];
            ga.ldb = Ki;
            ga.M = batch;
            ga.N = Ki;
            ga.K = No;
            ga.C = n->dz[1 - cur];
            ga.Ab = n->dzb[1 - cur];
            ga.Zmask = n->Z[l - 1];
            ga.ldc = Ki;
            gemm<false, true, EPI_DA>(ga, s);
            cur = 1 - cur;
        }
    }
    MK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_mlp_backward(fargo_mlp *n, const float *x, const float *t, int batch, float *loss)
{
    if (!n || !x || !t || batch < 1) return FARGO_ERR_BADARG;
    if (batch > n->max_batch) return FARGO_ERR_SIZE;
    return backward(n, x, t, batch, loss);
}

static int adam(fargo_mlp *n)
{
    k_adam_tick<<<1, 1, 0, n->stream>>>(n->hyper);
    k_adam<<<blocks_for(n->np, 256), 256, 0, n->stream>>>(n->w, n->m, n->v, n->g, n->wb, n->np, n->hyper, n->lt);
    MK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_mlp_adam(fargo_mlp *n) { return n ? adam(n) : FARGO_ERR_BADARG; }

extern "C" int fargo_mlp_train_step(fargo_mlp *n, const float *x, const float *t, int batch, float *loss)
{
    if (!n || !x || !t || batch < 1) return FARGO_ERR_BADARG;
    if (batch > n->max_batch) return FARGO_ERR_SIZE;
    const void *key[4] = {x, t, loss, nullptr};
    if (!n->gexec || memcmp(key, n->gkey, sizeof(key)) != 0 || n->gbatch != batch) {
        if (n->gexec) {
            cudaGraphExecDestroy(n->gexec);
            n->gexec = nullptr;
        }
        MK(cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal));
        int rc = backward(n, x, t, batch, loss);
        if (!rc) rc = adam(n);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(n->stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return FARGO_ERR_CUDA;
        e = cudaGraphInstantiate(&n->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return FARGO_ERR_CUDA;
        memcpy(n->gkey, key, sizeof(key));
        n->gbatch = batch;
    }
    MK(cudaGraphLaunch(n->gexec, n->stream));
    return FARGO_OK;
}

extern "C" int fargo_mlp_status(fargo_mlp *n)
{
    if (!n) return FARGO_ERR_BADARG;
    int h = 0;
    MK(cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    MK(cudaStreamSynchronize(n->stream));
    return h ? FARGO_ERR_BARRIER_TIMEOUT : FARGO_OK;
}

extern "C" int fargo_mlp_ensemble(const float *ys, int k, int batch, int n, float *mean, float *spread, void *stream)
{
    if (!ys || !mean || !spread || k < 2 || batch < 1 || n < 1) return FARGO_ERR_BADARG;
    k_ensemble<<<batch, 256, 0, (cudaStream_t)stream>>>(ys, k, batch, n, mean, spread);
    MK(cudaGetLastError());
    return FARGO_OK;
}
