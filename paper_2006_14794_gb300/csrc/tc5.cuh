// Fifth-generation tensor-core helpers (tcgen05, sm_100 family): operands in
// shared memory as K-major "core matrices" without swizzle, the accumulator
// in tensor memory (TMEM), completion signalled through an mbarrier.
//
// Layout of an R x K operand tile (K in 32-bit elements, a multiple of 8):
// element (r, k) at byte (r / 8) * SBO + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4,
// with SBO = (K / 4) * 128: each 8-row x 16-byte core matrix is 128
// contiguous bytes, core matrices adjacent in K are 128 bytes apart (LBO),
// those adjacent in rows SBO apart.  The MMA of k-step s (8 elements) starts
// at byte s * 256 of the tile.
//
// Split-TF32 products: x = hi + lo with hi = x rounded to TF32 and lo = the
// rest rounded to TF32; hi*hi + hi*lo + lo*hi keeps FP32 accuracy (the
// dropped lo*lo is below FP32 rounding), where one TF32 product would lose
// about 3e-4 relative.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sigk {
namespace tc5 {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__host__ __device__ constexpr int cm_off(int r, int k, int K) {
    return (r >> 3) * (K / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start, leading (K) and stride (row) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t desc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major
__host__ __device__ constexpr unsigned idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(void *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

// whole warp; the TMEM address is written to *slot (shared memory)
__device__ __forceinline__ void alloc(unsigned *slot, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(unsigned tmem, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(void *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bounded wait for the given phase parity; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(void *mbar, unsigned parity, long long max_iter) {
    unsigned done = 0;
    for (long long it = 0; it < max_iter && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return done != 0;
}

// 32 consecutive fp32 columns of this thread's TMEM lane (the warp reads lanes
// 32 * (warp % 4) ..); waits for the load
__device__ __forceinline__ void ld32(unsigned addr, float (&v)[32]) {
    unsigned r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// K of a d-channel operand: 4-channel groups, rounded up to whole k-steps of 8
__host__ __device__ inline int tc5_k_of(int64_t d) { return (int)(((d + 3) / 4 * 4 + 7) / 8 * 8); }

// Half of an operand row (K/8 float4 groups from k4 = half * K/8), scaled by
// s, split into TF32 hi and lo parts and stored into the K-major tiles
// (two threads per row; K <= 64).
__device__ __forceinline__ void store_half(unsigned char *hi, unsigned char *lo, int r, int half, int K,
                                           const float4 (&v)[8], float s) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i >= K / 8) break;
        const int k4 = half * (K / 8) + i;
        const float e[4] = {v[i].x * s, v[i].y * s, v[i].z * s, v[i].w * s};
        uint4 hh, ll;
        hh.x = tf32(e[0]); ll.x = tf32(e[0] - __uint_as_float(hh.x));
        hh.y = tf32(e[1]); ll.y = tf32(e[1] - __uint_as_float(hh.y));
        hh.z = tf32(e[2]); ll.z = tf32(e[2] - __uint_as_float(hh.z));
        hh.w = tf32(e[3]); ll.w = tf32(e[3] - __uint_as_float(hh.w));
        const int off = cm_off(r, 4 * k4, K);
        *reinterpret_cast<uint4 *>(hi + off) = hh;
        *reinterpret_cast<uint4 *>(lo + off) = ll;
    }
}

// D (+)= A B^T over K (M x K and N x K tiles, hi and lo parts): three MMAs per
// k-step.  One thread issues.
__device__ __forceinline__ void gemm_split(unsigned tmem, const unsigned char *ah, const unsigned char *al,
                                           const unsigned char *bh, const unsigned char *bl, int K, unsigned idesc,
                                           bool accumulate) {
    const unsigned sbo = (unsigned)(K / 4) * 128;
    bool acc = accumulate;
    for (int ks = 0; ks < K / 8; ++ks) {
        const unsigned off = (unsigned)ks * 256;
        const uint64_t dah = desc(smem_u32(ah) + off, 128, sbo), dal = desc(smem_u32(al) + off, 128, sbo);
        const uint64_t dbh = desc(smem_u32(bh) + off, 128, sbo), dbl = desc(smem_u32(bl) + off, 128, sbo);
        mma_tf32(tmem, dah, dbh, idesc, acc ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
        acc = true;
    }
}

}  // namespace tc5
}  // namespace sigk
