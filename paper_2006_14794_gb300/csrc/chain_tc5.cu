// The chain rule of the band backward on the fifth-generation tensor cores.
//
// The adjoint sweep leaves dk/dc for every coarse cell (Gbar, dense).  Since
// c(p, q) = 1/2 4^-lambda <dx_p, dy_q> (Sec. 3.1, remark after the scheme),
// the increments' gradients are the contractions
//   d dx = Gbar dy,      d dy = Gbar^T dx
// (times 1/2 4^-lambda, applied later), over every pair of a Gram at once:
// M = K = (paths x coarse intervals), N = d channels.
//
// One CTA owns a 128-row tile of the output and walks K in 32-deep chunks.
//  * Loads: every thread copies its share of chunk c + P - 1 (Gbar rows or
//    columns, and the increments) into a ring of P raw chunks in shared
//    memory with cp.async, so P - 1 chunks of HBM reads are in flight while
//    chunk c is worked on.
//  * Split: the threads read chunk c back, split each value x into TF32 parts
//    (PARTS = 2: x ~ h + m, 22 of FP32's 24 bits, products h h + h m + m h;
//    PARTS = 3: x = h + m + l exactly, six products down to 2^-33) and store
//    them as K-major core matrices into one of two MMA stages.
//  * MMAs: one thread issues the chunk's MMAs (D = 128 x N fp32) and commits
//    them to the stage's mbarrier (NS stages), which the stage's next fill,
//    NS chunks later, waits for.
//  * Accumulation: each chunk's MMAs accumulate in a TMEM region of their own
//    (NS + 1 in rotation).  The tensor core's accumulate is not a round-to-
//    nearest FP32 add: thousands of them into one tile bias a Gram's
//    contraction by about 1e-4 of the gradient.  Warps 0-3 read chunk c - NS's
//    region back (tcgen05.ld) once its mbarrier has completed, and the chunk
//    sums add up in FP32 registers.  The sum is written (or added) to C.
// Each CTA reads its 128 rows of Gbar once: the contraction is bound by
// reading Gbar from HBM, where the FP32-pipe kernel is bound by its FMAs.
//
// Waits are bounded: on expiry the block records SIGK_ETIMEOUT, gives its
// MMAs in flight one more bounded wait, frees its tensor memory and returns.
#include "sigk_internal.cuh"
#include "tc5.cuh"

namespace sigk {

namespace {

constexpr int CG_M = 128;    // rows of a tile: TMEM lanes
constexpr int CG_KC = 32;    // K per chunk: four k-steps of 8
constexpr int CG_T = 256;    // threads

// MMA stage: PARTS A parts (128 x 32), then PARTS B parts (NP x 32)
template <int PARTS>
__host__ __device__ inline int cg_stage_bytes(int NP) { return PARTS * (CG_M + NP) * CG_KC * 4; }
// raw chunk: A (128 rows of CG_RS floats, or 32 rows of 128) and B (32 x NP
// floats).  CG_RS = 36: 16-byte row pieces of 8 consecutive rows fall in 8
// distinct bank quads.
constexpr int CG_RS = CG_KC + 4;
__host__ __device__ inline int cg_raw_bytes(int NP) { return (CG_M * CG_RS + NP * CG_KC) * 4; }
template <int PARTS, int NS, int P>
__host__ __device__ inline int cg_smem_bytes(int NP) { return NS * cg_stage_bytes<PARTS>(NP) + P * cg_raw_bytes(NP); }

template <int PARTS>
__device__ __forceinline__ void split_parts(float x, unsigned (&p)[3]) {
    p[0] = tc5::tf32(x);
    const float r = x - __uint_as_float(p[0]);
    p[1] = tc5::tf32(r);
    p[2] = 0u;
    if constexpr (PARTS == 3) p[2] = tc5::tf32(r - __uint_as_float(p[1]));
}

__device__ __forceinline__ void cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc5::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc5::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct CgArgs {
    ChainGemm g;
    int NP;                  // N padded to 16, 32 or 64
    int *status;
    long long max_wait;
};

// NS: MMA stages (the wait for a stage is for the MMAs of chunk c - NS);
// P: raw chunks in the copy ring
template <int PARTS, int NS, int P>
__global__ void __launch_bounds__(CG_T, 1) chain_gemm_tc5_kernel(CgArgs a) {
    constexpr int CG_NR = NS + 1;   // TMEM regions: NS chunks in flight, one read back
    extern __shared__ __align__(1024) unsigned char cgs[];
    __shared__ __align__(8) unsigned long long mbar[NS];
    __shared__ unsigned tslot;
    const ChainGemm &g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NP = a.NP;
    const int64_t r0 = (int64_t)blockIdx.x * CG_M;
    // this tile's K range; a symmetric Gram's blocks below the diagonal are
    // zero and skipped (in whole chunks)
    int64_t kmin = 0, kmax = g.K;
    if (g.tri_rb > 0) {
        if (!g.trans) kmin = (r0 / g.tri_rb) * g.tri_cb;
        else {
            const int64_t rl = (r0 + CG_M - 1 < g.M ? r0 + CG_M - 1 : g.M - 1);
            kmax = (rl / g.tri_cb + 1) * g.tri_rb;
            if (kmax > g.K) kmax = g.K;
        }
    }
    const int64_t cfirst = kmin / CG_KC;
    const int nch = (int)((kmax + CG_KC - 1) / CG_KC - cfirst);
    // TMEM: CG_NR regions of RS columns, chunk c accumulating in region c % CG_NR
    const int RS = NP <= 32 ? 32 : 64;
    const int ncols = CG_NR * RS <= 128 ? 128 : (CG_NR * RS <= 256 ? 256 : 512);

    if (tid == 0)
        for (int q = 0; q < NS; ++q) tc5::mbar_init(&mbar[q]);
    if (warp == 0) tc5::alloc(&tslot, ncols);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const unsigned tmem = tslot;
    const unsigned idesc = tc5::idesc_tf32(CG_M, NP);

    unsigned char *stage0 = cgs;
    unsigned char *raw0 = cgs + NS * cg_stage_bytes<PARTS>(NP);
    auto a_part = [&](int s, int p) { return stage0 + s * cg_stage_bytes<PARTS>(NP) + p * (CG_M * CG_KC * 4); };
    auto b_part = [&](int s, int p) {
        return stage0 + s * cg_stage_bytes<PARTS>(NP) + PARTS * (CG_M * CG_KC * 4) + p * (NP * CG_KC * 4);
    };
    // raw chunk in slot q: A as [row][k] (trans = 0) or [k][row] (trans = 1),
    // then B as [k][n] with rows of NP floats
    auto raw_a = [&](int q) { return reinterpret_cast<float *>(raw0 + q * cg_raw_bytes(NP)); };
    auto raw_b = [&](int q) { return raw_a(q) + CG_M * CG_RS; };

    // ---- copies of chunk c into raw slot c % P.  trans = 0: thread (row
    // tid / 2, 16 K from (tid % 2) 16); trans = 1: thread (k tid / 8, 16 rows
    // from (tid % 8) 16).  B: thread (k tid / 8, NP / 8 channels).  Elements
    // outside the matrix are zeroed with plain stores (the same barrier that
    // publishes the copies publishes them).
    const bool avec = (g.g_ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(g.G) & 15) == 0);
    auto copy = [&](int c) {
        const int q = c % P;
        const int64_t kc = (cfirst + c) * CG_KC;
        float *ra = raw_a(q);
        if (!g.trans) {
            const int r = tid >> 1, k0 = (tid & 1) * 16;
            const int64_t gr = r0 + r;
            const float *src = g.G + gr * g.g_ld + kc + k0;
            float *dst = ra + r * CG_RS + k0;
            if (avec && gr < g.M && kc + k0 + 16 <= kmax) {
#pragma unroll
                for (int i = 0; i < 4; ++i) cp16(dst + 4 * i, src + 4 * i);
            } else {
#pragma unroll 4
                for (int j = 0; j < 16; ++j) {
                    if (gr < g.M && kc + k0 + j < kmax) cp4(dst + j, src + j);
                    else dst[j] = 0.f;
                }
            }
        } else {
            const int kk = tid >> 3, rs = (tid & 7) * 16;
            const int64_t k = kc + kk;
            const float *src = g.G + k * g.g_ld + r0 + rs;
            float *dst = ra + kk * CG_M + rs;
            if (avec && k < kmax && r0 + rs + 16 <= g.M) {
#pragma unroll
                for (int i = 0; i < 4; ++i) cp16(dst + 4 * i, src + 4 * i);
            } else {
#pragma unroll 4
                for (int j = 0; j < 16; ++j) {
                    if (k < kmax && r0 + rs + j < g.M) cp4(dst + j, src + j);
                    else dst[j] = 0.f;
                }
            }
        }
        // B: thread (channel tid % NP, K from (tid / NP) NP / 8): consecutive
        // threads copy consecutive channels
        const int n = tid % NP, kq = (tid / NP) * (NP >> 3);
        float *rb = raw_b(q);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= (NP >> 3)) break;
            const int64_t k = kc + kq + j;
            float *dst = rb + (kq + j) * NP + n;
            if (n < g.N && k < kmax) cp4(dst, g.Bm + k * g.N + n);
            else *dst = 0.f;
        }
    };

    // ---- split of raw chunk c into MMA stage s: thread (row ar, K half ah) of
    // A, rows fastest (a shared-memory phase of 8 lanes covers 8 rows);
    // thread (channel tid % NP, its copy's K) of B
    const int ar = tid & (CG_M - 1);
    const int ah = tid >> 7;
    auto split = [&](int c, int s) {
        const float *ra = raw_a(c % P);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float e[4];
            if (!g.trans) {
                const float4 v = *reinterpret_cast<const float4 *>(ra + ar * CG_RS + ah * 16 + 4 * i);
                e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) e[j] = ra[(ah * 16 + 4 * i + j) * CG_M + ar];
            }
            unsigned pp[4][3];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_parts<PARTS>(e[j], pp[j]);
            const int off = tc5::cm_off(ar, ah * 16 + 4 * i, CG_KC);
#pragma unroll
            for (int p = 0; p < PARTS; ++p)
                *reinterpret_cast<uint4 *>(a_part(s, p) + off) = make_uint4(pp[0][p], pp[1][p], pp[2][p], pp[3][p]);
        }
        const int n = tid % NP, kq = (tid / NP) * (NP >> 3);
        const float *rb = raw_b(c % P);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= (NP >> 3)) break;
            unsigned pp[3];
            split_parts<PARTS>(rb[(kq + j) * NP + n], pp);
            const int off = tc5::cm_off(n, kq + j, CG_KC);
#pragma unroll
            for (int p = 0; p < PARTS; ++p) *reinterpret_cast<unsigned *>(b_part(s, p) + off) = pp[p];
        }
    };

    // ---- the chunk's MMAs (one thread): the kept products of the parts.
    // Descriptors are the first stage's plus the byte offset / 16 (the start
    // address field counts 16-byte units; every offset is a multiple of 16).
    const uint64_t dbase = tc5::desc(tc5::smem_u32(stage0), 128, (unsigned)(CG_KC / 4) * 128);
    const unsigned sbytes = (unsigned)cg_stage_bytes<PARTS>(NP);
    const unsigned bpart0 = PARTS * (CG_M * CG_KC * 4), bpart = (unsigned)(NP * CG_KC * 4);
    auto issue = [&](int s, int region) {
        const unsigned d = tmem + (unsigned)(region * RS);
        constexpr int NPROD = PARTS == 3 ? 6 : 3;
        // (A part, B part): h h, h m, m h (, m m, h l, l h)
        constexpr int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
        const uint64_t ds = dbase + (((unsigned)s * sbytes) >> 4);
#pragma unroll
        for (int ks = 0; ks < CG_KC / 8; ++ks) {
#pragma unroll
            for (int t = 0; t < NPROD; ++t) {
                const uint64_t da = ds + ((pa[t] * (CG_M * CG_KC * 4) + ks * 256) >> 4);
                const uint64_t db = ds + ((bpart0 + pb[t] * bpart + ks * 256) >> 4);
                tc5::mma_tf32(d, da, db, idesc, (ks | t) ? 1u : 0u);   // each chunk starts its region afresh
            }
        }
    };

    unsigned phase[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) phase[q] = 0u;
    bool failed = false;
    // waits for the MMAs that last read stage s (block-uniform result)
    auto wait_stage = [&](int s) {
        const bool ok = tc5::mbar_wait(&mbar[s], phase[s], a.max_wait);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.status, (int)SIGK_ETIMEOUT);
            return false;
        }
        phase[s] ^= 1u;
        return true;
    };
    // chunk c's sum, read from its TMEM region into FP32 registers (warps 0-3:
    // the 128 rows), where the chunks add up with round-to-nearest
    float accr[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) accr[j] = 0.f;
    auto readback = [&](int c) {
        if (warp >= 4) return;
        tc5::fence_after();
        const unsigned base = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((c % CG_NR) * RS);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h * 32 < NP) {
                float v[32];
                tc5::ld32(base + (unsigned)(h * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) accr[h * 32 + j] += v[j];
            }
        }
        tc5::fence_before();
    };

    // chunks 0 .. P - 2 in flight before the loop, one group each
#pragma unroll
    for (int c = 0; c < P - 1; ++c) {
        if (c < nch) copy(c);
        cp_commit();
    }
    int issued[NS];   // commits on each stage not yet waited for
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = 0;
    for (int c = 0; c < nch; ++c) {
        const int s = c % NS;
        // chunk c + P - 1 into the raw slot that chunk c - 1 used
        if (c + P - 1 < nch) copy(c + P - 1);
        cp_commit();
        cp_wait<P - 1>();   // this thread's copies of chunk c have landed
        if (issued[s]) {
            // chunk c - NS read this stage: its MMAs are done (the wait's
            // barrier also publishes every thread's copies of chunk c)
            if (!wait_stage(s)) { failed = true; break; }
            issued[s] = 0;
            readback(c - NS);
        } else {
            __syncthreads();
        }
        split(c, s);
        tc5::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            issue(s, c % CG_NR);
            tc5::commit(&mbar[s]);
        }
        issued[s] = 1;
    }
    cp_wait<0>();
    // the last NS chunks, in order
    for (int c = nch >= NS ? nch - NS : 0; c < nch && !failed; ++c) {
        const int s = c % NS;
        if (!issued[s]) continue;
        if (!wait_stage(s)) { failed = true; break; }
        issued[s] = 0;
        readback(c);
    }
    if (failed) {
        // after a timeout, the MMAs in flight get one more bounded wait
        // before the accumulators are released; the result is not written
        for (int s = 0; s < NS; ++s)
            if (issued[s]) tc5::mbar_wait(&mbar[s], phase[s], a.max_wait);
    } else if (warp < 4) {
        const int64_t r = r0 + warp * 32 + lane;
        if (r < g.M) {
            float *dst = g.C + r * g.N;
#pragma unroll
            for (int j = 0; j < 64; ++j)
                if (j < g.N) dst[j] = g.add ? dst[j] + accr[j] : accr[j];
        }
    }
    tc5::fence_before();
    __syncthreads();
    if (warp == 0) tc5::dealloc(tmem, ncols);
}

// operand parts: 2 (three products a k-step; the chunked FP32 accumulation
// keeps the result at FP32 accuracy)
constexpr int CG_PARTS = 2;

template <int NS, int P>
cudaError_t cg_launch(const CgArgs &a, int64_t grid, cudaStream_t st) {
    auto kern = chain_gemm_tc5_kernel<CG_PARTS, NS, P>;
    const int smem = cg_smem_bytes<CG_PARTS, NS, P>(a.NP);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, CG_T, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool chain_gemm_tc5_ok(int64_t M, int64_t K, int N) { return N >= 1 && N <= 64 && M >= 1 && K >= 1; }

cudaError_t launch_chain_gemm_tc5(const ChainGemm &g, int *status, cudaStream_t st) {
    if (g.M <= 0) return cudaSuccess;
    CgArgs a;
    a.g = g;
    // N padded to 16, 32 or 64: the copies and splits deal the 32 x NP
    // increments of a chunk to 256 threads as (channel, K run), which needs NP
    // to divide 256
    a.NP = g.N <= 16 ? 16 : (g.N <= 32 ? 32 : 64);
    a.status = status;
    a.max_wait = 1LL << 26;
    const int64_t grid = (g.M + CG_M - 1) / CG_M;
    // three MMA stages and three raw chunks (a fourth stage measured no faster)
    return cg_launch<3, 3>(a, grid, st);
}

}  // namespace sigk
