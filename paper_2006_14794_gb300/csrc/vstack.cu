// Forward sweep, FP32, for pairs of uneven lengths with the increment Gram
// formed inside the sweep: no coefficient ever reaches global memory.
//
// The scheme (Sec. 3.1, explicit finite differences on P_lambda) in the
// difference form of fwd_chain.cu:
//   Q(a,b) = Q(a-1,b) + c (K(a,b-1) + K(a-1,b)),   K(a,b) = K(a,b-1) + Q(a,b),
//   c = 1/2 4^-lambda <dx_p, dy_q>                (remark after the scheme),
// swept along anti-diagonals (Sec. 3.1.1).
//
// Layout of the work.  Each pair's rows refine its shorter path.  A thread
// block solves a chain of pairs whose shorter paths need the same number NW of
// bands of 64 coarse rows ("stack" of NW warps; the stack is padded at the top
// with zero-increment rows, where K = 1 and Q = 0 exactly).  Warp w owns band
// w; lane l of it owns two coarse rows, i.e. R = 2 * 2^lambda refined rows, and
// sweeps them as one warp of the register chain (fwd_chain.cu): row r of lane
// l works on column t - R l - r at step t, rows turn over to the chain's next
// pair when they leave a pair's last column, so the pipeline fills once per
// chain.  Band w runs DM macro-steps (of R steps) behind band w - 1 and takes
// its top input, the bottom row of band w - 1 (one (K, Q) a step), from a
// 64-slot ring in shared memory (band 0 reads a ring of boundary values
// (1, 0), and the bottom band writes a ring nobody reads, so every warp runs
// the same code).  A block barrier every 16 refined steps orders that
// hand-off: a value is written one barrier period before it is read, and its
// slot is written again only two periods later.
//
// Coefficients.  A lane keeps its two coarse rows' increments in registers
// and forms every coarse-cell coefficient it enters as a d-term dot product
// (FFMA2 over channel pairs), shared by the cell's 4^lambda refined cells.
// Group 0 of a lane enters chain column J at a window, group 1 the column
// group 0 entered one window before, so a window reads one column increment
// (d floats) from shared memory and the two alternate between two register
// sets.  The column increments of the chain sit in a ring in shared memory
// indexed by the chain column (the pairs' columns one after another, left
// virtual columns zero), which one producer warp fills with cp.async VS_F
// barrier periods ahead; the ring holds every column between the stack's
// first and last rows' wavefronts.  Window 0 of a lane always reads an even
// chain column and window 1 an odd one, at the same index (the lane's macro-
// step), so the ring keeps even and odd columns apart, each column padded to
// an odd number of 16-byte units: the 32 lanes, one column apart, then read
// distinct bank quads with one address a macro-step.  A lane's row
// increments for its next pair wait in a 2-row slot of shared memory, fetched
// by the lane itself with cp.async when it enters the current pair.
//
// The increments themselves, x[p+1] - x[p] for every point row of the call,
// are formed once by vs_inc_kernel into the workspace (16-byte rows of
// channel quads, zero-padded), so that every later copy is a plain 16-byte
// cp.async; those of the X side are scaled by 1/2 4^-lambda there (a power
// of two: exact), so every pair, whichever side its rows refine, forms
// c = <dx, dy> with exactly one factor scaled.  Planning happens on the
// device from the offsets (no host round trip; a CUDA graph replays it for
// any lengths up to max_len):
//   vs_pairs_kernel: per pair, orientation, stack height, macro-steps T;
//   vs_plan_kernel (one block): pairs sorted by (stack height, T descending),
//     the number of chains of each height chosen so that every chain ends at
//     about the same time with all of them resident in three quarters of the
//     register file, pairs dealt to chains in snake order;
//   vstack_kernel, one launch per stack height on library streams.
#include <string.h>

#include <mutex>

#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int VS_NG = 2;       // coarse rows per lane = windows per macro-step
constexpr int VS_NWMAX = 8;    // bands (warps) per stack: shorter paths of <= 513 points
constexpr int VS_F = 4;        // column fill distance, in barrier periods
constexpr int VS_P = 16;       // refined steps per barrier period
constexpr int VS_HS = 64;      // hand-off slots (>= 2 VS_P + 1), a power of two dividing 32 R
constexpr int VS_RS = VS_HS + 1;   // hand-off ring entries: slots at entries 1 .. 64 (entry 64 is slot 0)
constexpr int VS_PT = 1024;    // threads of the planning block
constexpr int VS_MAXREG = 112; // registers a thread: 18 warps a SM

struct VsPair {
    int64_t rows, cols;        // increment rows of the row (shorter) path and the column path
    int64_t out0;              // output slot
    int T, vrows, nqv, cls;    // macro-steps, virtual coarse rows (top) and columns (left); NW - 1 (-1: k = 1)
};
struct VsEntry {               // a pair in chain order
    int64_t rows, cols, out0;
    int T, vrows, nqv, pad;
};
struct VsClass {
    int count, start;          // pairs of the stack height, their first index in order[]
    int nch, chain0;           // chains, global index of the first
    unsigned long long work;   // sum of T over the pairs
};

struct VsArgs {
    PairSrc src;
    float *out;
    float4 *inc;               // [2 capA][D4] increments: the launch's X rows, then its Y rows at capA
    int64_t capA;
    VsPair *plan;
    int *order;                // pair ids sorted by stack height, then T descending
    int *hist;                 // [VS_NWMAX * TK] counts, then scatter cursors
    VsClass *cls;              // [VS_NWMAX]
    int *chain_off;            // [chains + 1] first entry of each chain
    VsEntry *ent;              // [n] the chains' pairs
    int64_t n;
    int lam, TK, D4, cap_warps;
    float scale;               // 1/2 4^-lambda
};

// Macro-steps per barrier period, and the delay of band w + 1 behind band w.
__host__ __device__ constexpr int vs_bm(int lam) { return VS_P / (VS_NG << lam); }
__host__ __device__ constexpr int vs_dm(int lam) { return 32 + vs_bm(lam); }
// Columns of the chain ring of a stack of nw bands: the span between the
// wavefronts of the top band's lane 0 and the bottom band's lane 31, plus the
// columns in flight (the fill runs VS_F periods ahead), in multiples of 8.
__host__ __device__ inline int vs_rc(int lam, int nw) {
    const int v = ((VS_F + 1) * vs_bm(lam) + (nw - 1) * vs_dm(lam) + 32) * VS_NG;
    return (v + 7) / 8 * 8;
}
// 16-byte units a ring column takes: D4 padded to an odd count, so that lanes
// reading consecutive entries hit distinct bank quads.
__host__ __device__ constexpr int vs_es(int D4) { return D4 == 4 ? 5 : (D4 == 2 ? 3 : 1); }
__host__ __device__ inline int64_t vs_smem(int lam, int nw, int D4) {
    return (int64_t)vs_rc(lam, nw) * vs_es(D4) * 16 + (int64_t)nw * 32 * VS_NG * D4 * 16 +
           (int64_t)(nw + 1) * VS_RS * 8;
}

// 16 bytes global -> shared, asynchronously; zeros when !valid.
// D4 consecutive 16-byte units global -> shared, asynchronously; zeros when !valid.
template <int D4>
__device__ __forceinline__ void vs_cp_row(void *dst, const void *src, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(src), "r"(n) : "memory");
    if constexpr (D4 >= 2)
        asm volatile("cp.async.cg.shared.global [%0+16], [%1+16], 16, %2;" ::"r"(s), "l"(src), "r"(n) : "memory");
    if constexpr (D4 >= 4) {
        asm volatile("cp.async.cg.shared.global [%0+32], [%1+32], 16, %2;" ::"r"(s), "l"(src), "r"(n) : "memory");
        asm volatile("cp.async.cg.shared.global [%0+48], [%1+48], 16, %2;" ::"r"(s), "l"(src), "r"(n) : "memory");
    }
}
__device__ __forceinline__ void vs_cp16(void *dst, const void *src, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void vs_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void vs_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// <x, y> over D4 channel quads, FFMA2 over channel pairs.
template <int D4>
__device__ __forceinline__ float vs_dot(const float4 (&x)[D4], const float4 (&y)[D4]) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int c4 = 0; c4 < D4; ++c4) {
        acc = __ffma2_rn(make_float2(x[c4].x, x[c4].y), make_float2(y[c4].x, y[c4].y), acc);
        acc = __ffma2_rn(make_float2(x[c4].z, x[c4].w), make_float2(y[c4].z, y[c4].w), acc);
    }
    return acc.x + acc.y;
}

// ---- increments and planning ---------------------------------------------

// Channels c .. c + 3 of x[p + 1] - x[p] (x points at row p), channels >= d zero.
__device__ __forceinline__ float4 vs_inc4(const float *x, int64_t d, int64_t c) {
    float e[4] = {0.f, 0.f, 0.f, 0.f};
    if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(x + c));
        const float4 v = __ldg(reinterpret_cast<const float4 *>(x + d + c));
        return make_float4(v.x - u.x, v.y - u.y, v.z - u.z, v.w - u.w);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (c + k < d) e[k] = __ldg(x + d + c + k) - __ldg(x + c + k);
    return make_float4(e[0], e[1], e[2], e[3]);
}

// Every point row of the launch's X range (rows a_off[kbase] .. a_off[kbase+n])
// and Y range gets its increment to the next row; the last row of each range
// has none, and rows that straddle two paths are never read.
__global__ void vs_inc_kernel(VsArgs a) {
    const int64_t d = a.src.d;
    const int D4 = a.D4;
    const int64_t a0 = a.src.a_off[a.src.kbase], a1 = a.src.a_off[a.src.kbase + a.n];
    const int64_t b0 = a.src.b_off[a.src.kbase], b1 = a.src.b_off[a.src.kbase + a.n];
    const int64_t na = a1 - a0 > 1 ? a1 - a0 - 1 : 0, nb = b1 - b0 > 1 ? b1 - b0 - 1 : 0;
    const int64_t tot = (na + nb) * D4;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < tot;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = v / D4;
        const int c4 = (int)(v - r * D4);
        const bool isb = r >= na;
        const int64_t rr = isb ? r - na : r;
        const float *x = (const float *)(isb ? a.src.B : a.src.A) + ((isb ? b0 : a0) + rr) * d;
        float4 e = vs_inc4(x, d, 4 * (int64_t)c4);
        if (!isb) e = make_float4(e.x * a.scale, e.y * a.scale, e.z * a.scale, e.w * a.scale);
        a.inc[((isb ? a.capA : 0) + rr) * D4 + c4] = e;
    }
}

__global__ void vs_pairs_kernel(VsArgs a) {
    const int64_t a0 = a.src.a_off[a.src.kbase], b0 = a.src.b_off[a.src.kbase];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const PairRef pr = pair_ref(a.src, k);
        VsPair p;
        memset(&p, 0, sizeof(p));
        p.cls = -1;
        p.out0 = pr.out0;
        if (pr.la < 2 || pr.lb < 2) {
            a.out[pr.out0] = 1.f;   // a single point: k = 1
            a.plan[k] = p;
            continue;
        }
        const bool sw = pr.la > pr.lb;
        const int64_t ia = pr.a_row0 - a0, ib = a.capA + pr.b_row0 - b0;
        p.rows = sw ? ib : ia;
        p.cols = sw ? ia : ib;
        const int lr = (int)(sw ? pr.lb : pr.la), lc = (int)(sw ? pr.la : pr.lb);
        int nw = (lr - 1 + 32 * VS_NG - 1) / (32 * VS_NG);
        if (nw > VS_NWMAX) nw = VS_NWMAX;   // cannot happen: the host checks max_len
        int T = lc / 2;                     // ceil((lc - 1) / VS_NG) coarse columns per macro-step
        if (T < 2) T = 2;
        if (T > a.TK - 1) T = a.TK - 1;     // cannot happen either (TK bounds T)
        p.T = T;
        p.cls = nw - 1;
        p.vrows = 32 * VS_NG * nw - (lr - 1);
        p.nqv = VS_NG * T - (lc - 1);
        a.plan[k] = p;
        atomicAdd(&a.hist[p.cls * a.TK + (a.TK - 1 - T)], 1);
    }
}

// Exclusive scan of v[0 .. n) in place by one block (a multiple of 32
// threads, at most 1024); sh holds 33 values.  Returns the total.
__device__ int vs_block_scan(int *v, int64_t n, int *sh) {
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5, nwp = nt >> 5;
    const int64_t per = (n + nt - 1) / nt;
    const int64_t q0 = (int64_t)t * per < n ? (int64_t)t * per : n, q1 = q0 + per < n ? q0 + per : n;
    int s = 0;
    for (int64_t i = q0; i < q1; ++i) s += v[i];
    int x = s;   // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int wv = lane < nwp ? sh[lane] : 0;
        int inc = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < nwp) sh[lane] = inc - wv;
        if (lane == 31) sh[32] = inc;
    }
    __syncthreads();
    int run = sh[wid] + x - s;
    for (int64_t i = q0; i < q1; ++i) { const int y = v[i]; v[i] = run; run += y; }
    const int total = sh[32];
    __syncthreads();
    return total;
}

// Pairs of chain ch (of W) of a class of cnt pairs dealt in snake order.
__device__ __forceinline__ int vs_chain_len(int ch, int W, int cnt) {
    const int full = cnt / W, rem = cnt - full * W;
    return full + (((full & 1) ? (W - 1 - ch) : ch) < rem ? 1 : 0);
}

__global__ void __launch_bounds__(VS_PT) vs_plan_kernel(VsArgs a) {
    __shared__ int shi[33];
    __shared__ unsigned long long swork[VS_NWMAX];
    __shared__ int schain0[VS_NWMAX + 1], snch[VS_NWMAX], sstart[VS_NWMAX + 1], smaxT[VS_NWMAX];
    const int t = threadIdx.x;
    if (t < VS_NWMAX) { swork[t] = 0; smaxT[t] = 0; }
    // 1. sort by (stack height, T descending): scan the histogram, scatter
    const int nkeys = VS_NWMAX * a.TK;
    const int nsorted = vs_block_scan(a.hist, nkeys, shi);
    if (t < VS_NWMAX) sstart[t] = a.hist[t * a.TK];
    if (t == 0) sstart[VS_NWMAX] = nsorted;
    __syncthreads();
    for (int64_t k = t; k < a.n; k += blockDim.x) {
        const VsPair &p = a.plan[k];
        if (p.cls < 0) continue;
        const int slot = atomicAdd(&a.hist[p.cls * a.TK + (a.TK - 1 - p.T)], 1);
        a.order[slot] = (int)k;
        atomicAdd(&swork[p.cls], (unsigned long long)p.T);
        atomicMax(&smaxT[p.cls], p.T);
    }
    __syncthreads();
    // 2. chains per height: the smallest makespan tau (in macro-steps, a chain
    //    of sum T taking sum T + 32 + (NW - 1) DM) whose chains all fit in
    //    cap_warps resident warps (NW + 1 a chain); found by two rounds of
    //    evaluating one candidate tau a thread
    __shared__ long long slo, shi2;
    __shared__ int sbest;
    const long long DM = vs_dm(a.lam);
    if (t == 0) {
        long long lo = 0, hi = 0;
        for (int c = 0; c < VS_NWMAX; ++c) {
            if (sstart[c + 1] == sstart[c]) continue;
            const long long ovh = 32 + c * DM;
            lo = lo > ovh + smaxT[c] ? lo : ovh + smaxT[c];
            const long long h = ovh + (long long)swork[c];
            hi = hi > h ? hi : h;
        }
        slo = lo;
        shi2 = hi;
    }
    auto chains = [&](long long tau, int c) -> long long {
        const long long cnt = sstart[c + 1] - sstart[c];
        const long long room = tau - 32 - c * DM;
        long long m = room > 0 ? ((long long)swork[c] + room - 1) / room : cnt;
        if (m > cnt) m = cnt;
        return m < 1 ? 1 : m;
    };
    auto fits = [&](long long tau) {
        long long w = 0;
        for (int c = 0; c < VS_NWMAX; ++c)
            if (sstart[c + 1] > sstart[c]) w += chains(tau, c) * (c + 2);
        return w <= a.cap_warps;
    };
    for (int round = 0; round < 2; ++round) {
        if (t == 0) sbest = (int)blockDim.x;
        __syncthreads();
        const long long lo = slo, hi = shi2, span = hi - lo;
        const long long tau = lo + span * t / ((long long)blockDim.x - 1);
        if (fits(tau)) atomicMin(&sbest, t);
        __syncthreads();
        if (t == 0) {
            const int k = sbest;
            if (k < (int)blockDim.x) {   // tau_k fits, tau_(k-1) does not
                shi2 = lo + span * k / ((long long)blockDim.x - 1);
                if (k > 0) slo = lo + span * (k - 1) / ((long long)blockDim.x - 1) + 1;
            } else {
                slo = hi;                // nothing fits: one chain a height
            }
            if (slo > shi2) slo = shi2;
        }
        __syncthreads();
    }
    if (t == 0) {
        const long long tau = shi2;
        int g = 0;
        for (int c = 0; c < VS_NWMAX; ++c) {
            const int cnt = sstart[c + 1] - sstart[c];
            const int m = cnt == 0 ? 0 : (int)chains(tau, c);
            VsClass ci;
            ci.count = cnt;
            ci.start = sstart[c];
            ci.nch = m;
            ci.chain0 = g;
            ci.work = swork[c];
            a.cls[c] = ci;
            snch[c] = m;
            schain0[c] = g;
            g += m;
        }
        schain0[VS_NWMAX] = g;
    }
    __syncthreads();
    const int nchains = schain0[VS_NWMAX];
    // 3. chain offsets
    for (int gc = t; gc < nchains; gc += blockDim.x) {
        int c = 0;
        while (gc >= schain0[c + 1]) ++c;
        a.chain_off[gc] = vs_chain_len(gc - schain0[c], snch[c], sstart[c + 1] - sstart[c]);
    }
    if (t == 0) a.chain_off[nchains] = 0;
    __syncthreads();
    vs_block_scan(a.chain_off, nchains + 1, shi);
    // 4. every pair's entry: sorted position s of height c is the jj-th pair
    //    of chain ch
    for (int s = t; s < nsorted; s += blockDim.x) {
        int c = 0;
        while (s >= sstart[c + 1]) ++c;
        const int si = s - sstart[c], W = snch[c];
        const int jj = si / W, r = si - jj * W;
        const int ch = (jj & 1) ? W - 1 - r : r;
        const VsPair &p = a.plan[a.order[s]];
        VsEntry e;
        e.rows = p.rows;
        e.cols = p.cols;
        e.out0 = p.out0;
        e.T = p.T;
        e.vrows = p.vrows;
        e.nqv = p.nqv;
        e.pad = 0;
        a.ent[a.chain_off[schain0[c] + ch] + jj] = e;
    }
}

// ---- the stack sweep ----------------------------------------------------------
// One block per chain of stack height NW = c + 1: warps 0 .. NW-1 sweep, warp
// NW fills the column ring.  Every warp runs the same number of barrier
// periods.
template <int LAM, int D4, bool IMPL>
__global__ void __maxnreg__(VS_MAXREG) vstack_kernel(VsArgs a, int c) {
    constexpr int S = 1 << LAM;
    constexpr int R = VS_NG * S;     // refined rows per lane
    constexpr int H = R / 2;         // rows i and i + H share a float2 (groups 0 and 1)
    constexpr int JOUT = R - 2;      // step of the corner in a turn-over macro-step
    constexpr int BM = vs_bm(LAM), DM = vs_dm(LAM);
    constexpr int ES = vs_es(D4);
    static_assert(BM >= 1 && BM * R == VS_P, "barrier period: whole macro-steps");
    extern __shared__ __align__(16) float4 vsm[];

    const VsClass ci = a.cls[c];
    if ((int)blockIdx.x >= ci.nch) return;   // whole block
    const int NW = c + 1;
    const int RC = vs_rc(LAM, NW), RC2 = RC / 2;
    float4 *ring = vsm;                                          // even columns, then odd: RC x ES
    float4 *slots = ring + RC * ES;                              // NW x 32 lanes x 2 rows x D4
    // hand-off rings: ring w is band w's top input, ring w + 1 its bottom row
    // (ring 0 holds the boundary (1, 0), ring NW is never read)
    float2 *hand = reinterpret_cast<float2 *>(slots + NW * 32 * VS_NG * D4);   // (NW + 1) x VS_RS
    const int gc = ci.chain0 + blockIdx.x;
    const int e0 = a.chain_off[gc];
    const int np = a.chain_off[gc + 1] - e0;
    const VsEntry *ent = a.ent + e0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int tsum = 0;
    for (int j = lane; j < np; j += 32) tsum += ent[j].T;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(FULL, tsum, o);
    const int total_m = tsum + 32;                 // the chain plus lane 31's lag
    const int NPER = (total_m + (NW - 1) * DM + BM - 1) / BM;

    for (int u = threadIdx.x; u < RC * ES; u += blockDim.x) ring[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u = threadIdx.x; u < VS_RS; u += blockDim.x) hand[u] = make_float2(1.f, 0.f);
    __syncthreads();

    if (warp == NW) {
        // ---- producer: chain columns J = q * PER + cu of period q, unit u =
        // lane + 32 k of the period's PER x D4 (column cu = u / D4, channel
        // quad u mod D4); each unit keeps its own cursor over the chain's
        // pairs.  Column J sits at entry (J & 1) RC2 + (J >> 1) mod RC2.
        constexpr int PER = BM * VS_NG;
        constexpr int NU = (PER * D4 + 31) / 32;   // units a lane
        static_assert(NU <= 2, "a lane fills at most two units a period");
        bool act[NU];
        int cu[NU], c4u[NU], jr[NU], j[NU], Tc[NU], nq[NU], Tn[NU], nqn[NU];
        long long C[NU];
        int64_t cb[NU], cbn[NU];
        float4 *base[NU];
#pragma unroll
        for (int k = 0; k < NU; ++k) {
            const int u = lane + 32 * k, c4 = u % D4;
            act[k] = u < PER * D4;
            cu[k] = u / D4;
            c4u[k] = c4;
            jr[k] = cu[k] >> 1;   // ring entry (within its parity) of the unit's column
            base[k] = ring + ((cu[k] & 1) ? RC2 * ES : 0) + c4;
            j[k] = 0;
            C[k] = 0;             // chain column of pair j's column 0
            Tc[k] = ent[0].T; nq[k] = ent[0].nqv; cb[k] = ent[0].cols;
            Tn[k] = 0; nqn[k] = 0; cbn[k] = 0;
            if (np > 1) { Tn[k] = ent[1].T; nqn[k] = ent[1].nqv; cbn[k] = ent[1].cols; }
        }
        auto issue = [&](int q) {
#pragma unroll
            for (int k = 0; k < NU; ++k) {
                if (!act[k]) continue;
                const long long J = (long long)q * PER + cu[k];
                while (j[k] < np && J >= C[k] + (long long)Tc[k] * VS_NG) {
                    C[k] += (long long)Tc[k] * VS_NG;
                    ++j[k];
                    Tc[k] = Tn[k]; nq[k] = nqn[k]; cb[k] = cbn[k];
                    if (j[k] + 1 < np) {
                        const VsEntry &e = ent[j[k] + 1];
                        Tn[k] = e.T; nqn[k] = e.nqv; cbn[k] = e.cols;
                    }
                }
                bool valid = false;
                const float4 *src = a.inc;
                if (j[k] < np) {
                    const long long qi = J - C[k] - nq[k];
                    if (qi >= 0) { valid = true; src = a.inc + (cb[k] + qi) * D4 + c4u[k]; }
                }
                vs_cp16(base[k] + jr[k] * ES, src, valid);
                jr[k] += PER / 2;
                if (jr[k] >= RC2) jr[k] -= RC2;
            }
            vs_commit();
        };
        for (int q = 0; q < VS_F; ++q) issue(q);
        vs_wait<VS_F - 1>();
        __syncthreads();
        for (int p = 0; p < NPER; ++p) {
            issue(p + VS_F);
            vs_wait<VS_F - 1>();   // period p + 1's columns have landed
            __syncthreads();
        }
        vs_wait<0>();
        return;
    }

    // ---- sweep warps
    float4 *slot = slots + (warp * 32 + lane) * VS_NG * D4;
    const float2 *hin = hand + warp * VS_RS;
    float2 *hout = hand + (warp + 1) * VS_RS;
    const int prow0 = (warp * 32 + lane) * VS_NG;   // the lane's first coarse row of the stack
    auto fetch_rows = [&](int64_t rows, int vr, bool any) {
        const int pr = prow0 - vr;
        const float4 *src = a.inc + (rows + pr) * D4;
        vs_cp_row<D4>(slot, any && pr >= 0 ? (const void *)src : (const void *)a.inc, any && pr >= 0);
        vs_cp_row<D4>(slot + D4, any && pr + 1 >= 0 ? (const void *)(src + D4) : (const void *)a.inc,
                      any && pr + 1 >= 0);
        vs_commit();
    };
    fetch_rows(ent[0].rows, ent[0].vrows, true);
    int64_t rn = 0;
    int vrn = 0;
    if (np > 1) { rn = ent[1].rows; vrn = ent[1].vrows; }
    // lane cursor: pair cj of the chain, macro-step pos in it (negative before
    // the chain), T of this pair and the next, output slots of this pair and
    // the one before
    int cj = 0, pos = -lane, T = ent[0].T, Tn = np > 1 ? ent[1].T : 1;
    long long ocur = ent[0].out0, oprev = -1;

    float2 KP[H], QP[H];             // (K, Q) of rows (i, i + H)
    float2 C2[2];                    // coefficients of groups (0, 1) entered in window 0 / 1
    float4 dxr[VS_NG][D4], Y2[2][D4];   // row increments; group 0's column of window 0 / 1
#pragma unroll
    for (int i = 0; i < H; ++i) { KP[i] = make_float2(1.f, 1.f); QP[i] = make_float2(0.f, 0.f); }
    C2[0] = make_float2(0.f, 0.f);
    C2[1] = C2[0];
#pragma unroll
    for (int c4 = 0; c4 < D4; ++c4) {
        dxr[0][c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        dxr[1][c4] = dxr[0][c4];
        Y2[0][c4] = dxr[0][c4];
        Y2[1][c4] = dxr[0][c4];
    }
    float pK = 1.f, pQ = 0.f;
    int qr = (RC2 - lane % RC2) % RC2;   // ring entry of the lane's macro-step (-lane at the start)
    __syncthreads();   // the producer's first columns

    for (int p = 0; p < NPER; ++p) {
#pragma unroll 1
        for (int b = 0; b < BM; ++b) {
            const int ml = p * BM + b - warp * DM;   // the warp's macro-step
            if (ml < 0 || ml >= total_m) continue;
            if (ml == 0 && lane == 0) { const float2 h = hin[VS_HS]; pK = h.x; pQ = h.y; }   // slot 0
            // hand-off slot of step t = ml R + j: entry hb + 1 + j, hb = ml R mod VS_HS (no
            // wrap: hb <= VS_HS - R); the band above wrote it at its own step t + 32 R,
            // the same entry since VS_HS divides 32 R
            const float2 *hi = hin + ((ml * R) & (VS_HS - 1));
            float2 *ho = hout + ((ml * R) & (VS_HS - 1));
            const bool trans = pos == 0;
            if (trans) vs_wait<0>();   // this pair's rows are in the slot
            const float4 *ye = ring + qr * ES;
            qr = qr + 1 == RC2 ? 0 : qr + 1;
#pragma unroll
            for (int w = 0; w < VS_NG; ++w) {
                // group 0 enters chain column 2 mm + w (even / odd half of the ring)
#pragma unroll
                for (int c4 = 0; c4 < D4; ++c4) Y2[w][c4] = ye[w * RC2 * ES + c4];
                if (trans) {
                    // group w's rows start the pair in this window
#pragma unroll
                    for (int c4 = 0; c4 < D4; ++c4) dxr[w][c4] = slot[w * D4 + c4];
                }
                {
                    // group 1 takes the column group 0 entered one window before
                    float c0 = vs_dot<D4>(dxr[0], Y2[w]);
                    float c1 = vs_dot<D4>(dxr[1], Y2[1 - w]);
                    if constexpr (IMPL) {
                        c0 = scheme_coef(c0, SIGK_SCHEME_IMPLICIT);
                        c1 = scheme_coef(c1, SIGK_SCHEME_IMPLICIT);
                    }
                    C2[w] = make_float2(c0, c1);
                }
#pragma unroll
                for (int jj = 0; jj < S; ++jj) {
                    const int jstep = w * S + jj;
                    const float kH1 = KP[H - 1].x, qH1 = QP[H - 1].x;   // row H-1 before this step
                    float shK = 0.f, shQ = 0.f;
#pragma unroll
                    for (int i = H - 1; i >= 0; --i) {
                        const int s1 = i % S;                // rows i (group 0) and i + H (group 1)
                        if (jj == s1 && trans) {            // row starts its next pair now: k(.,0) = 1
                            if (w == 0) KP[i].x = 1.f;
                            else KP[i].y = 1.f;
                        }
                        const float2 cf = (jj >= s1) ? C2[w] : C2[1 - w];
                        float2 ku, qu;
                        if (i > 0) {
                            ku = KP[i > 0 ? i - 1 : 0];
                            qu = QP[i > 0 ? i - 1 : 0];
                        } else {
                            ku = make_float2(pK, kH1);
                            qu = make_float2(pQ, qH1);
                        }
                        const float2 sum = __fadd2_rn(KP[i], ku);
                        const float2 qn = __ffma2_rn(cf, sum, qu);
                        KP[i] = __fadd2_rn(KP[i], qn);
                        QP[i] = qn;
                        if (i == H - 1) {
                            shK = __shfl_up_sync(FULL, KP[i].y, 1);
                            shQ = __shfl_up_sync(FULL, QP[i].y, 1);
                            // the stack's last row just finished the previous pair's last column
                            if (jstep == JOUT && trans && lane == 31 && warp == NW - 1 && cj >= 1 && cj <= np)
                                a.out[oprev] = KP[i].y;
                            // the band's bottom row: the band below reads it as its top input
                            if (lane == 31) ho[1 + jstep] = make_float2(KP[i].y, QP[i].y);
                        }
                    }
                    {
                        const float2 h = hi[1 + jstep];
                        pK = (lane == 0) ? h.x : shK;
                        pQ = (lane == 0) ? h.y : shQ;
                    }
                }
            }
            if (trans) {
                // the slot is free: the next pair's rows (zeros past the chain)
                fetch_rows(rn, vrn, cj + 1 < np);
                if (cj + 2 < np) { rn = ent[cj + 2].rows; vrn = ent[cj + 2].vrows; }
            }
            if (++pos == T && cj < np) {
                pos = 0;
                ++cj;
                T = Tn;
                Tn = cj + 1 < np ? ent[cj + 1].T : 1;
                oprev = ocur;
                ocur = cj < np ? ent[cj].out0 : -1;
            }
        }
        __syncthreads();
    }
    vs_wait<0>();
}

// Instances: dyadic orders 0-2 (2, 4, 8 refined rows a lane), d <= 4, 8, 16.
#define SIGK_VSTACK_CASES(X) \
    X(0, 1) X(0, 2) X(0, 4) X(1, 1) X(1, 2) X(1, 4) X(2, 1) X(2, 2) X(2, 4)

template <int LAM, int D4, bool IMPL>
cudaError_t vs_prepare(int smem_max, int *regs) {
    auto kern = vstack_kernel<LAM, D4, IMPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    *regs = fa.numRegs;
    return cudaSuccess;
}

template <int LAM, int D4, bool IMPL>
cudaError_t vs_launch(const VsArgs &a, int c, int grid, int smem, cudaStream_t st) {
    vstack_kernel<LAM, D4, IMPL><<<grid, (c + 2) * 32, smem, st>>>(a, c);
    return cudaGetLastError();
}

int vs_d4(int64_t d) {
    const int q = (int)((d + 3) / 4);
    return q == 3 ? 4 : q;
}

struct VsLayout {
    int64_t plan, order, hist, cls, chain_off, ent, inc, total;
};

int64_t vs_up256(int64_t v) { return (v + 255) / 256 * 256; }

int vs_tk(int64_t max_len) {
    const int64_t t = max_len / 2;
    return (int)((t < 2 ? 2 : t) + 1);
}

VsLayout vs_layout(int64_t n, int64_t max_len, int64_t d) {
    VsLayout L;
    int64_t o = 256;   // a 256-byte header: the status word sigk_stream_status reads (no waits here: 0)
    L.plan = o; o = vs_up256(o + n * (int64_t)sizeof(VsPair));
    L.order = o; o = vs_up256(o + n * 4);
    L.hist = o; o = vs_up256(o + (int64_t)VS_NWMAX * vs_tk(max_len) * 4);
    L.cls = o; o = vs_up256(o + VS_NWMAX * (int64_t)sizeof(VsClass));
    L.chain_off = o; o = vs_up256(o + (n + 1) * 4);
    L.ent = o; o = vs_up256(o + n * (int64_t)sizeof(VsEntry));
    L.inc = o; o = vs_up256(o + 2 * n * max_len * vs_d4(d) * 16);
    L.total = o;
    return L;
}

// The stack heights' sweeps run concurrently on library-owned streams, forked
// from and joined back to the caller's stream by events (a stream capture
// records them as a forked graph).  Created once per device, on first use.
struct VsStreams {
    bool ok;
    cudaStream_t s[VS_NWMAX];
    cudaEvent_t pre, inc, fork, join[VS_NWMAX];
};
constexpr int VS_MAX_DEVICES = 64;
std::mutex g_vs_mu;
VsStreams g_vs[VS_MAX_DEVICES];

cudaError_t vs_streams(int dev, VsStreams **out) {
    if (dev < 0 || dev >= VS_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_vs_mu);
    VsStreams &v = g_vs[dev];
    if (!v.ok) {
        cudaError_t e = cudaEventCreateWithFlags(&v.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v.pre, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v.inc, cudaEventDisableTiming);
        for (int c = 0; c < VS_NWMAX && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&v.s[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v.join[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
        v.ok = true;
    }
    *out = &v;
    return cudaSuccess;
}

}  // namespace

bool vstack_supported(int lam, int64_t d, int64_t max_len, int dtype, int kernel) {
    return dtype == SIGK_F32 && kernel == SIGK_KERNEL_LINEAR && lam >= 0 && lam <= 2 && d >= 1 &&
           d <= 16 && max_len >= 1 && max_len - 1 <= 32LL * VS_NG * VS_NWMAX;
}

int64_t vstack_workspace_bytes(int64_t n, int64_t max_len, int64_t d) {
    return n <= 0 ? 0 : vs_layout(n, max_len, d).total;
}

cudaError_t launch_vstack(const PairSrc &src, int64_t n, int lam, int64_t max_len, float *out, void *ws,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0, maxthr = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&maxthr, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return e;
    const int D4 = vs_d4(src.d);
    const bool impl = src.scheme == SIGK_SCHEME_IMPLICIT;
    const VsLayout L = vs_layout(n, max_len, src.d);
    unsigned char *w = (unsigned char *)ws;
    VsArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.out = out;
    a.inc = (float4 *)(w + L.inc);
    a.capA = n * max_len;
    a.plan = (VsPair *)(w + L.plan);
    a.order = (int *)(w + L.order);
    a.hist = (int *)(w + L.hist);
    a.cls = (VsClass *)(w + L.cls);
    a.chain_off = (int *)(w + L.chain_off);
    a.ent = (VsEntry *)(w + L.ent);
    a.n = n;
    a.lam = lam;
    a.TK = vs_tk(max_len);
    a.D4 = D4;
    a.scale = 0.5f / (float)(1 << (2 * lam));
    // resident warps the planner may fill: the register file's share, a warp
    // at a time (allocation in 256-register units) -
    const int smem_max = (int)vs_smem(lam, VS_NWMAX, D4);
    int regs = 0;
    bool found = false;
#define X(l, dd)                                                                                \
    if (lam == l && D4 == dd) {                                                                 \
        e = impl ? vs_prepare<l, dd, true>(smem_max, &regs) : vs_prepare<l, dd, false>(smem_max, &regs); \
        found = true;                                                                           \
    }
    SIGK_VSTACK_CASES(X)
#undef X
    if (!found) return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    const int per_warp = ((regs * 32 + 255) / 256) * 256;
    int wps = per_warp > 0 ? 65536 / per_warp : 1;
    if (wps > maxthr / 32) wps = maxthr / 32;
    // three quarters of it: chains of several stack heights share the SMs, and
    // a block that finds no room runs in a second wave
    a.cap_warps = sms * wps * 3 / 4;
    if (a.cap_warps < 2 * (VS_NWMAX + 1)) a.cap_warps = 2 * (VS_NWMAX + 1);

    if ((e = cudaMemsetAsync(w, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.hist, 0, (size_t)VS_NWMAX * a.TK * 4, st)) != cudaSuccess) return e;
    VsStreams *vs = nullptr;
    if ((e = vs_streams(dev, &vs)) != cudaSuccess) return e;
    // the increments (bandwidth-bound) on a side stream while one block plans
    if ((e = cudaEventRecord(vs->pre, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(vs->s[0], vs->pre, 0)) != cudaSuccess) return e;
    const int64_t iun = 2 * n * max_len * D4;
    const int igrid = (int)((iun + 255) / 256 < (int64_t)sms * 8 ? (iun + 255) / 256 : (int64_t)sms * 8);
    vs_inc_kernel<<<igrid > 0 ? igrid : 1, 256, 0, vs->s[0]>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(vs->inc, vs->s[0])) != cudaSuccess) return e;
    const int pgrid = (int)((n + 255) / 256 < (int64_t)sms * 4 ? (n + 255) / 256 : (int64_t)sms * 4);
    vs_pairs_kernel<<<pgrid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    vs_plan_kernel<<<1, VS_PT, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(vs->fork, st)) != cudaSuccess) return e;
    for (int c = 0; c < VS_NWMAX; ++c) {
        cudaStream_t sc = vs->s[c];
        if ((e = cudaStreamWaitEvent(sc, vs->fork, 0)) != cudaSuccess) return e;
        if (c > 0 && (e = cudaStreamWaitEvent(sc, vs->inc, 0)) != cudaSuccess) return e;
        // the planner gives height c at most min(pairs, cap / (c + 2)) chains
        int64_t grid = a.cap_warps / (c + 2);
        if (grid > n) grid = n;
        if (grid < 1) grid = 1;
        const int smem = (int)vs_smem(lam, c + 1, D4);
        found = false;
#define X(l, dd)                                                                                   \
        if (lam == l && D4 == dd) {                                                                \
            e = impl ? vs_launch<l, dd, true>(a, c, (int)grid, smem, sc)                           \
                     : vs_launch<l, dd, false>(a, c, (int)grid, smem, sc);                         \
            found = true;                                                                          \
        }
        SIGK_VSTACK_CASES(X)
#undef X
        if (!found) return cudaErrorInvalidValue;
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(vs->join[c], sc)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, vs->join[c], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sigk
