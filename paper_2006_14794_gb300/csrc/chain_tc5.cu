// The chain rule of the band backward on the fifth-generation tensor cores.
//
// The adjoint sweep leaves dk/dc for every coarse cell (Gbar, dense).  Since
// c(p, q) = 1/2 4^-lambda <dx_p, dy_q> (Sec. 3.1, remark after the scheme),
// the increments' gradients are the contractions
//   d dx = Gbar dy,      d dy = Gbar^T dx
// (times 1/2 4^-lambda, applied later), over every pair of a Gram at once:
// M = K = (paths x coarse intervals), N = d channels.  Here one CTA owns a
// 128-row tile of the output and walks K in 32-deep chunks: 256 threads load
// the next chunk of Gbar and of the increments into registers while the MMAs
// of the current one run, then split each value exactly into three TF32
// parts, x = h + m + l (11 + 11 + 2 significant bits), and store them into
// K-major core matrices in shared memory (two stages).  One thread issues the
// chunk's MMAs, six per k-step (h h + h m + m h + m m + h l + l h: the dropped
// terms are below 2^-33 relative), with D = 128 x N fp32 in TMEM, and commits
// them to the stage's mbarrier, which the stage's next fill waits for.  (Two
// parts, h + m, keep only 22 of FP32's 24 bits: over the tens of thousands of
// terms of a Gram's contraction, with terms of both signs, that loses about
// 1e-4 of the gradient.)  A chunk accumulates in a TMEM region of its own
// (three in rotation): the tensor core's accumulate is not a round-to-nearest
// FP32 add, and thousands of them into one tile bias the sum by about 1e-4,
// so each chunk's 24 MMAs stay in their region, which warps 0-3 read back
// (tcgen05.ld) two chunks later, once its mbarrier has completed, and add into
// FP32 registers; the sum is then written (or added) to C.  Each CTA reads its 128
// rows of Gbar once: the contraction is bound by reading Gbar from HBM, where
// the FP32-pipe kernel it replaces was bound by its FMAs.
//
// Waits are bounded: on expiry the block records SIGK_ETIMEOUT, gives its
// MMAs in flight one more bounded wait, frees its tensor memory and returns.
#include "sigk_internal.cuh"
#include "tc5.cuh"

namespace sigk {

namespace {

constexpr int CG_M = 128;    // rows of a tile: TMEM lanes
constexpr int CG_KC = 32;    // K per stage: four k-steps of 8
constexpr int CG_T = 256;    // threads

constexpr int CG_PARTS = 3;   // TF32 parts of each operand
constexpr int CG_NR = 3;      // TMEM accumulator regions: chunks c, c - 1 in flight, c - 2 read back

__host__ __device__ inline int cg_stage_bytes(int NP) {
    return CG_PARTS * CG_M * CG_KC * 4 + CG_PARTS * NP * CG_KC * 4;
}

// x = h + m + l exactly, each part a TF32 value
__device__ __forceinline__ void split3(float x, unsigned &h, unsigned &m, unsigned &l) {
    h = tc5::tf32(x);
    const float r = x - __uint_as_float(h);
    m = tc5::tf32(r);
    l = tc5::tf32(r - __uint_as_float(m));
}

struct CgArgs {
    ChainGemm g;
    int NP;                  // N padded to a multiple of 16
    int *status;
    long long max_wait;
};

__global__ void __launch_bounds__(CG_T, 1) chain_gemm_tc5_kernel(CgArgs a) {
    extern __shared__ __align__(1024) unsigned char cgs[];
    __shared__ __align__(8) unsigned long long mbar[2];
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
    const int ncols = NP <= 32 ? 128 : 256;

    if (tid == 0) {
        tc5::mbar_init(&mbar[0]);
        tc5::mbar_init(&mbar[1]);
    }
    if (warp == 0) tc5::alloc(&tslot, ncols);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const unsigned tmem = tslot;
    const unsigned idesc = tc5::idesc_tf32(CG_M, NP);

    // A rows: trans = 0, thread (row tid / 2, half tid % 2) reads 16
    // consecutive K of its row; trans = 1, thread (row tid % 128, half
    // tid / 128) reads 16 K of its column of Gbar (consecutive threads read
    // consecutive rows: coalesced)
    const int ar = g.trans ? (tid & (CG_M - 1)) : (tid >> 1);
    const int ah = g.trans ? (tid >> 7) : (tid & 1);
    const bool avec = !g.trans && (g.g_ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(g.G) & 15) == 0);
    // B: thread (kk = tid / 8, n = (tid % 8) NP/8 ..) reads NP/8 channels
    const int bk = tid >> 3, bn0 = (tid & 7) * (NP >> 3);
    float4 av[8];
    float bv[8];
    auto fetch = [&](int c) {
        const int64_t k0 = (cfirst + c) * CG_KC + ah * 16;
        const int64_t r = r0 + ar;
        if (!g.trans) {
            const float *src = g.G + r * g.g_ld + k0;
            if (avec && r < g.M && k0 + 16 <= kmax) {
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = __ldcs(reinterpret_cast<const float4 *>(src) + i);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float e[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int64_t k = k0 + 4 * i + j;
                        e[j] = (r < g.M && k < kmax) ? __ldcs(src + 4 * i + j) : 0.f;
                    }
                    av[i] = make_float4(e[0], e[1], e[2], e[3]);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float e[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t k = k0 + 4 * i + j;
                    e[j] = (r < g.M && k < kmax) ? __ldcs(g.G + k * g.g_ld + r) : 0.f;
                }
                av[i] = make_float4(e[0], e[1], e[2], e[3]);
            }
        }
        const int64_t kb = (cfirst + c) * CG_KC + bk;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = bn0 + j;
            bv[j] = (j < (NP >> 3) && n < g.N && kb < kmax) ? __ldg(g.Bm + kb * g.N + n) : 0.f;
        }
    };
    // stage s: A parts h, m, l (128 x 32 each), then B parts h, m, l (NP x 32)
    auto a_part = [&](int s, int p) { return cgs + s * cg_stage_bytes(NP) + p * (CG_M * CG_KC * 4); };
    auto b_part = [&](int s, int p) {
        return cgs + s * cg_stage_bytes(NP) + CG_PARTS * (CG_M * CG_KC * 4) + p * (NP * CG_KC * 4);
    };
    auto store = [&](int s) {
        unsigned char *a0 = a_part(s, 0), *a1 = a_part(s, 1), *a2 = a_part(s, 2);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int off = tc5::cm_off(ar, ah * 16 + 4 * i, CG_KC);
            const float e[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
            uint4 h, m, l;
            split3(e[0], h.x, m.x, l.x);
            split3(e[1], h.y, m.y, l.y);
            split3(e[2], h.z, m.z, l.z);
            split3(e[3], h.w, m.w, l.w);
            *reinterpret_cast<uint4 *>(a0 + off) = h;
            *reinterpret_cast<uint4 *>(a1 + off) = m;
            *reinterpret_cast<uint4 *>(a2 + off) = l;
        }
        unsigned char *b0 = b_part(s, 0), *b1 = b_part(s, 1), *b2 = b_part(s, 2);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= (NP >> 3)) break;
            unsigned h, m, l;
            split3(bv[j], h, m, l);
            const int off = tc5::cm_off(bn0 + j, bk, CG_KC);
            *reinterpret_cast<unsigned *>(b0 + off) = h;
            *reinterpret_cast<unsigned *>(b1 + off) = m;
            *reinterpret_cast<unsigned *>(b2 + off) = l;
        }
    };
    // the chunk's MMAs: six products per k-step (one thread issues)
    auto issue = [&](int s, int region) {
        const unsigned sbo = (unsigned)(CG_KC / 4) * 128;
        const unsigned d = tmem + (unsigned)(region * RS);
        bool acc = false;   // each chunk starts its region afresh
        // (A part, B part) of the kept products: h h, h m, m h, m m, h l, l h
        const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
        for (int ks = 0; ks < CG_KC / 8; ++ks) {
            const unsigned off = (unsigned)ks * 256;
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const uint64_t da = tc5::desc(tc5::smem_u32(a_part(s, pa[t])) + off, 128, sbo);
                const uint64_t db = tc5::desc(tc5::smem_u32(b_part(s, pb[t])) + off, 128, sbo);
                tc5::mma_tf32(d, da, db, idesc, acc ? 1u : 0u);
                acc = true;
            }
        }
    };
    unsigned phase[2] = {0u, 0u};
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

    if (nch > 0) fetch(0);
    int issued[2] = {0, 0};   // commits on each stage not yet waited for
    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        if (issued[s]) {
            // chunk c - 2 read this stage: its MMAs are done, its sum is read back
            if (!wait_stage(s)) { failed = true; break; }
            issued[s] = 0;
            readback(c - 2);
        }
        store(s);
        tc5::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            issue(s, c % CG_NR);
            tc5::commit(&mbar[s]);
        }
        issued[s] = 1;
        if (c + 1 < nch) fetch(c + 1);
    }
    // the last one or two chunks, in order
    for (int c = nch >= 2 ? nch - 2 : 0; c < nch && !failed; ++c) {
        const int s = c & 1;
        if (!issued[s]) continue;
        if (!wait_stage(s)) { failed = true; break; }
        issued[s] = 0;
        readback(c);
    }
    if (failed) {
        // after a timeout, the MMAs in flight get one more bounded wait
        // before the accumulators are released; the result is not written
        for (int s = 0; s < 2; ++s)
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

}  // namespace

bool chain_gemm_tc5_ok(int64_t M, int64_t K, int N) { return N >= 1 && N <= 64 && M >= 1 && K >= 1; }

cudaError_t launch_chain_gemm_tc5(const ChainGemm &g, int *status, cudaStream_t st) {
    if (g.M <= 0) return cudaSuccess;
    CgArgs a;
    a.g = g;
    a.NP = (g.N + 15) / 16 * 16;
    a.status = status;
    a.max_wait = 1LL << 26;
    const int smem = 2 * cg_stage_bytes(a.NP);
    cudaError_t e = cudaFuncSetAttribute(chain_gemm_tc5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (g.M + CG_M - 1) / CG_M;
    chain_gemm_tc5_kernel<<<(unsigned)grid, CG_T, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sigk
