// Forward sweep, FP32, for pairs of uneven lengths in the band form: the row
// chain of fwd_chain.cu / band.cu (one warp sweeps a chain of pairs, lane l
// owning refined rows R*l .. R*l+R-1 of a band of 32 R rows, the anti-diagonal
// wavefront of Sec. 3.1.1 held across the warp's registers, rows turning over
// to the chain's next pair so that the pipeline fills once per chain), with
// the difference form of the scheme of Sec. 3.1,
//   Q(a,b) = Q(a-1,b) + c (K(a,b-1) + K(a-1,b)),   K(a,b) = K(a,b-1) + Q(a,b),
// c = 1/2 4^-lambda <dx_p, dy_q> (remark after the scheme), and with every
// pair carrying its own geometry.
//
// Each pair's rows refine its shorter path.  A pair goes to the smallest band
// height class 32 R that holds its Ni refined rows (padding at the top with
// zero-increment rows, where K = 1 and Q = 0 exactly) and sweeps T macro-steps
// of R refined columns (padding at the left likewise).  All of this is planned
// on the device from the offsets, so one call needs no host round trip and can
// be captured in a CUDA graph:
//   1. vb_pairs_kernel: per pair, orientation, class, T, padding; a histogram
//      of (class, T);
//   2. vb_plan_kernel (one block): pairs sorted by class and T descending;
//      each class gets W chains (warps) and its pairs are dealt to them in a
//      snake order (longest first), which balances the chains' lengths; every
//      chain's coefficients are laid out contiguously;
//   3. per class, vb_coef_kernel: every coarse-cell coefficient of the class's
//      pairs into the band layout of band.cu (slot (pair, pos, lane) holds the
//      lane's NG x NG cells of macro-step pos as [window][group]; the cells a
//      pair's rows still need after the next pair started, w < g at pos 0,
//      live in the next pair's slot 0, and after a chain's last pair in one
//      extra slot);
//   4. per class, vband_sweep_kernel: the chained sweep, each lane streaming
//      its window rows through a cp.async ring in shared memory (a window row
//      is NG floats; the ring keeps VB_RING windows in flight).
#include <string.h>

#include <mutex>

#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int VB_WARPS = 2;    // warps per CTA of the sweep
constexpr int VB_RING = 8;     // coefficient windows in flight per lane
constexpr int VB_CT = 256;     // threads per CTA of the contraction
constexpr int VB_DC = 32;      // channels staged per pass of the contraction
constexpr int VB_PT = 1024;    // threads of the planning block
constexpr int VB_NCLS = 4;     // band height classes of one dyadic order at most

// Per-lane stride of a ring entry (floats): 16-byte rows padded so that the
// 8 lanes of a shared-memory phase of a 16-byte load hit distinct bank quads.
__host__ __device__ constexpr int vb_lane_stride(int NG) { return NG >= 8 ? NG + 4 : NG; }

struct VbPair {
    int64_t r_row0, c_row0;    // first point rows of the row (shorter) and column paths
    int lr, lc;                // their lengths
    int swapped;               // rows come from src.B (the Y paths)
    int cls;                   // band class; -1: a path with one point (k = 1)
    int T;                     // macro-steps
    int vrows, nqv;            // virtual coarse rows (top) and columns (left)
    int first, last;           // first / last pair of its chain
    int64_t base;              // float offset of the pair's slot 0 in the band
    int64_t out0;              // output slot
};

struct VbClassInfo {
    int count, start;          // pairs of the class, their first index in order[]
    int W, chain0;             // chains, global index of the first one
};

struct VbArgs {
    PairSrc src;
    float *out;
    float *band;
    VbPair *plan;
    int *order;                // pair ids sorted by class, then T descending
    int *hist;                 // [ncls * TK] counts, then scatter cursors
    VbClassInfo *cinfo;        // [VB_NCLS]
    int64_t *chain_base;       // [chains] float offset of each chain's first slot
    int *chain_off;            // [chains + 1] first entry of each chain in cpid / cT
    int *cpid, *cT;            // the chains' pairs in chain order, and their T
    int64_t *scan;             // [chains] scratch of the planner
    int64_t n;
    int lam, ncls, TK;
    int R[VB_NCLS];
    int cap[VB_NCLS];          // resident warps of each class's sweep
    float scale;               // 1/2 4^-lambda
};

__device__ __forceinline__ int vb_ng(const VbArgs &a, int c) { return a.R[c] >> a.lam; }

__global__ void vb_pairs_kernel(VbArgs a) {
    const int S = 1 << a.lam;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const PairRef pr = pair_ref(a.src, k);
        VbPair p;
        memset(&p, 0, sizeof(p));
        p.cls = -1;
        p.out0 = pr.out0;
        if (pr.la < 2 || pr.lb < 2) {
            a.out[pr.out0] = 1.f;   // a single point: k = 1
            a.plan[k] = p;
            continue;
        }
        p.swapped = pr.la > pr.lb;
        p.r_row0 = p.swapped ? pr.b_row0 : pr.a_row0;
        p.c_row0 = p.swapped ? pr.a_row0 : pr.b_row0;
        p.lr = (int)(p.swapped ? pr.lb : pr.la);
        p.lc = (int)(p.swapped ? pr.la : pr.lb);
        const int Ni = (p.lr - 1) * S, Nj = (p.lc - 1) * S;
        int c = 0;
        while (c < a.ncls && 32 * a.R[c] < Ni) ++c;
        if (c == a.ncls) c = a.ncls - 1;   // cannot happen: the host checks the longest path
        const int R = a.R[c];
        int T = (Nj + R - 1) / R;
        if (T < 2) T = 2;
        if (T > a.TK - 1) T = a.TK - 1;    // cannot happen either (TK bounds T)
        p.cls = c;
        p.T = T;
        p.vrows = (32 * R - Ni) / S;
        p.nqv = (T * R - Nj) / S;
        a.plan[k] = p;
        atomicAdd(&a.hist[c * a.TK + (a.TK - 1 - T)], 1);
    }
}

// Exclusive scan of v[0 .. n) in place by one block; returns the total (to
// every thread).
template <typename T>
__device__ T block_scan(T *v, int64_t n, T *sh) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int64_t per = (n + nt - 1) / nt, b0 = t * per, b1 = b0 + per < n ? b0 + per : n;
    T s = 0;
    for (int64_t i = b0; i < b1; ++i) s += v[i];
    sh[t] = s;
    __syncthreads();
    if (t == 0) {
        T run = 0;
        for (int i = 0; i < nt; ++i) { const T x = sh[i]; sh[i] = run; run += x; }
        sh[nt] = run;
    }
    __syncthreads();
    T run = sh[t];
    for (int64_t i = b0; i < b1; ++i) { const T x = v[i]; v[i] = run; run += x; }
    const T total = sh[nt];
    __syncthreads();
    return total;
}

// The chain's j-th pair in order[] (class start + the snake position).
__device__ __forceinline__ int64_t vb_snake(int j, int c, int W) {
    return (int64_t)j * W + ((j & 1) ? (W - 1 - c) : c);
}
__device__ __forceinline__ int vb_chain_len(int c, int W, int count) {
    const int full = count / W, rem = count - full * W;
    return full + (((full & 1) ? (W - 1 - c) : c) < rem ? 1 : 0);
}

__global__ void __launch_bounds__(VB_PT) vb_plan_kernel(VbArgs a) {
    __shared__ int64_t sh64[VB_PT + 1];
    __shared__ int shi[VB_PT + 1];
    __shared__ int sW[VB_NCLS], sChain0[VB_NCLS + 1];
    const int t = threadIdx.x;
    // 1. sort by (class, T descending): scan the histogram, scatter
    const int nkeys = a.ncls * a.TK;
    const int nsorted = block_scan<int>(a.hist, nkeys, shi);   // pairs with a class
    if (t < a.ncls) {
        const int s0 = a.hist[t * a.TK];
        const int s1 = t + 1 < a.ncls ? a.hist[(t + 1) * a.TK] : nsorted;
        a.cinfo[t].start = s0;
        a.cinfo[t].count = s1 - s0;
    }
    __syncthreads();
    for (int64_t k = t; k < a.n; k += blockDim.x) {
        const VbPair &p = a.plan[k];
        if (p.cls < 0) continue;
        const int slot = atomicAdd(&a.hist[p.cls * a.TK + (a.TK - 1 - p.T)], 1);
        a.order[slot] = (int)k;
    }
    __syncthreads();
    // 2. chains per class
    if (t == 0) {
        int g = 0;
        for (int c = 0; c < a.ncls; ++c) {
            const int cnt = a.cinfo[c].count;
            const int W = cnt == 0 ? 0 : (cnt < a.cap[c] ? cnt : a.cap[c]);
            a.cinfo[c].W = W;
            a.cinfo[c].chain0 = g;
            sW[c] = W;
            sChain0[c] = g;
            g += W;
        }
        sChain0[a.ncls] = g;
    }
    __syncthreads();
    const int nchains = sChain0[a.ncls];
    // 3. each chain's size in floats (its pairs' slots and one extra slot) and
    //    its number of pairs
    for (int gc = t; gc < nchains; gc += blockDim.x) {
        int c = 0;
        while (gc >= sChain0[c + 1]) ++c;
        const int ch = gc - sChain0[c], W = sW[c], cnt = a.cinfo[c].count, st = a.cinfo[c].start;
        const int ng = vb_ng(a, c);
        const int64_t slot = 32LL * ng * ng;
        const int np = vb_chain_len(ch, W, cnt);
        int64_t sz = slot;   // the extra slot after the chain's last pair
        for (int j = 0; j < np; ++j) sz += (int64_t)a.plan[a.order[st + vb_snake(j, ch, W)]].T * slot;
        a.scan[gc] = sz;
        a.chain_off[gc] = np;
    }
    if (t == 0) a.chain_off[nchains] = 0;
    __syncthreads();
    block_scan<int64_t>(a.scan, nchains, sh64);
    block_scan<int>(a.chain_off, nchains + 1, shi);
    // 4. every pair's slot-0 offset, the chains' pair lists
    for (int gc = t; gc < nchains; gc += blockDim.x) {
        int c = 0;
        while (gc >= sChain0[c + 1]) ++c;
        const int ch = gc - sChain0[c], W = sW[c], cnt = a.cinfo[c].count, st = a.cinfo[c].start;
        const int ng = vb_ng(a, c);
        const int64_t slot = 32LL * ng * ng;
        const int np = vb_chain_len(ch, W, cnt);
        int64_t base = a.scan[gc];
        a.chain_base[gc] = base;
        const int off = a.chain_off[gc];
        for (int j = 0; j < np; ++j) {
            const int pid = a.order[st + vb_snake(j, ch, W)];
            VbPair &p = a.plan[pid];
            p.base = base;
            p.first = j == 0;
            p.last = j == np - 1;
            a.cpid[off + j] = pid;
            a.cT[off + j] = p.T;
            base += (int64_t)p.T * slot;
        }
    }
}

// ---- coefficients: every coarse cell of a class's pairs into its chain's
// band.  A thread computes WQ windows x NG groups of one slot (lane l,
// position pos), each cell a d-term dot product of increments staged
// channel-major in shared memory (as band_coef_kernel, with each pair's own
// geometry).  Threads are numbered lane-fastest: the 32 threads of a warp are
// the 32 lanes of one (position, window quarter), so they read the same
// column increments (a broadcast) and their own row increments (rows padded
// to a conflict-free stride, vb_lane_stride).
// Channel strides of the staged increments: multiples of 4 floats (16-byte
// rows) that are 4 (mod 32), so the 8 channels a staging thread group writes
// land in 8 bank quads.
__host__ __device__ constexpr int vb_pad32(int n) { return ((n + 27) / 32) * 32 + 4; }
template <int NG>
__host__ __device__ constexpr int vb_xstride() { return vb_pad32(32 * vb_lane_stride(NG)); }
__host__ __device__ inline int vb_ystride(int T, int NG) { return vb_pad32(((T * NG + 2 * NG + 3) / 4) * 4); }
template <int NG>
__host__ __device__ constexpr int vb_gpos(int g) {   // groups g and g + NG/2 side by side
    return g < NG / 2 ? 2 * g : 2 * (g - NG / 2) + 1;
}

// n consecutive floats from 16-byte aligned shared memory (n % 4 == 0), or
// two (n == 2, 8-byte aligned)
template <int N>
__device__ __forceinline__ void vb_lds(float (&v)[N], const float *p) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int h = 0; h < N / 4; ++h) {
            const float4 t = *reinterpret_cast<const float4 *>(p + 4 * h);
            v[4 * h] = t.x; v[4 * h + 1] = t.y; v[4 * h + 2] = t.z; v[4 * h + 3] = t.w;
        }
    } else {
        static_assert(N == 2, "2 or a multiple of 4");
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
}

// Increments of channels c .. c + 3 at point row p (x points at row p):
// x[p + 1] - x[p], channels >= d zero.
__device__ __forceinline__ void vb_inc4(float (&e)[4], const float *x, int64_t d, int64_t c) {
    if ((d & 3) == 0 && c + 4 <= d && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(x + c));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(x + d + c));
        e[0] = b.x - a.x; e[1] = b.y - a.y; e[2] = b.z - a.z; e[3] = b.w - a.w;
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (c + k < d) e[k] = __ldg(x + d + c + k) - __ldg(x + c + k);
}

template <int NG, int WQ>
__global__ void __launch_bounds__(VB_CT) vb_coef_kernel(VbArgs a, int cls, int dc) {
    extern __shared__ __align__(16) float vcs[];
    constexpr int NPP = 32 * NG, XL = vb_lane_stride(NG), XS = vb_xstride<NG>(), SLOT = NG * NG;
    constexpr int NQW = NG / WQ;
    constexpr int YN = WQ + NG - 1, YL = (YN + 3) / 4 * 4;   // column increments a thread reads
    static_assert(NG == 2 ? WQ == 2 : WQ % 4 == 0, "vector loads of the column increments");
    const VbClassInfo ci = a.cinfo[cls];
    const int64_t d = a.src.d;
    float *dxs = vcs;
    float *dys = vcs + dc * XS;
    for (int t = blockIdx.x; t < ci.count; t += gridDim.x) {
        const int pid = a.order[ci.start + t];
        const VbPair p = a.plan[pid];
        const float *rows = (const float *)(p.swapped ? a.src.B : a.src.A) + p.r_row0 * d;
        const float *cols = (const float *)(p.swapped ? a.src.A : a.src.B) + p.c_row0 * d;
        const int nx = p.lr - 1, ny = p.lc - 1, T = p.T, NQ = T * NG;
        const int YS = vb_ystride(T, NG);
        const int nthr = 32 * (T + 1) * NQW;
        for (int b0 = 0; b0 < nthr; b0 += VB_CT) {
            const int u = b0 + (int)threadIdx.x;
            const int l = u & 31, pq = u >> 5;
            const int pos = pq / NQW, w0 = (pq - pos * NQW) * WQ;
            float acc[WQ][NG];
#pragma unroll
            for (int w = 0; w < WQ; ++w)
#pragma unroll
                for (int g = 0; g < NG; ++g) acc[w][g] = 0.f;
            for (int64_t c0 = 0; c0 < d; c0 += dc) {
                if (d > dc || b0 == 0) {
                    __syncthreads();
                    // four channels a thread: one 16-byte load per point when the
                    // rows allow it (d a multiple of 4), else scalar loads
                    const int dq = dc / 4;
                    for (int v = threadIdx.x; v < dq * NPP; v += VB_CT) {
                        const int P = v / dq, c = 4 * (v - (v / dq) * dq);
                        const int pr = P - p.vrows;
                        float e[4] = {0.f, 0.f, 0.f, 0.f};
                        if (pr >= 0 && pr < nx) vb_inc4(e, rows + (int64_t)pr * d, d, c0 + c);
                        float *o = dxs + c * XS + (P / NG) * XL + P % NG;
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[k * XS] = e[k];
                    }
                    for (int v = threadIdx.x; v < dq * YS; v += VB_CT) {
                        const int iq = v / dq, c = 4 * (v - (v / dq) * dq);
                        const int q = iq - (NG - 1) - p.nqv;   // real column
                        float e[4] = {0.f, 0.f, 0.f, 0.f};
                        if (q >= 0 && q < ny && iq - (NG - 1) < NQ) vb_inc4(e, cols + (int64_t)q * d, d, c0 + c);
                        float *o = dys + c * YS + iq;
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[k * YS] = e[k];
                    }
                    __syncthreads();
                }
                if (u < nthr) {
                    const int cn = (int)(d - c0 < dc ? d - c0 : dc);
#pragma unroll 2
                    for (int c = 0; c < cn; ++c) {
                        float xv[NG], yv[YL];
                        vb_lds<NG>(xv, dxs + c * XS + l * XL);
                        // index Q + NG - 1, Q = pos NG + w - g; 16-byte aligned for NG >= 4,
                        // 8-byte aligned (two float2) for NG = 2
                        const float *yr = dys + c * YS + pos * NG + w0;
                        if constexpr (NG >= 4) {
                            vb_lds<YL>(yv, yr);
                        } else {
                            const float2 y0 = *reinterpret_cast<const float2 *>(yr);
                            const float2 y1 = *reinterpret_cast<const float2 *>(yr + 2);
                            yv[0] = y0.x; yv[1] = y0.y; yv[2] = y1.x; yv[3] = y1.y;
                        }
#pragma unroll
                        for (int w = 0; w < WQ; ++w)
#pragma unroll
                            for (int g = 0; g < NG; ++g) acc[w][g] = fmaf(xv[g], yv[w - g + NG - 1], acc[w][g]);
                    }
                }
            }
            if (u >= nthr) continue;
            float *dst = a.band + p.base + ((int64_t)pos * 32 + l) * SLOT;   // pos = T: the next slot 0
            if (pos > 0 && pos < T) {
#pragma unroll
                for (int w = 0; w < WQ; ++w) {
                    float o[NG];
#pragma unroll
                    for (int g = 0; g < NG; ++g) o[vb_gpos<NG>(g)] = scheme_coef(acc[w][g] * a.scale, a.src.scheme);
                    if constexpr (NG % 4 == 0) {
#pragma unroll
                        for (int h = 0; h < NG / 4; ++h)
                            reinterpret_cast<float4 *>(dst + (w0 + w) * NG)[h] =
                                make_float4(o[4 * h], o[4 * h + 1], o[4 * h + 2], o[4 * h + 3]);
                    } else {
                        reinterpret_cast<float2 *>(dst + (w0 + w) * NG)[0] = make_float2(o[0], o[1]);
                    }
                }
                continue;
            }
#pragma unroll
            for (int w = 0; w < WQ; ++w)
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const int ww = w0 + w;
                    const float v = scheme_coef(acc[w][g] * a.scale, a.src.scheme);
                    float *o = dst + ww * NG + vb_gpos<NG>(g);
                    if (pos == 0) {
                        // the pair's own cells; the previous pair of the chain
                        // writes the cells w < g of this slot (its tail)
                        if (ww >= g) *o = v;
                        else if (p.first) *o = 0.f;
                    } else {
                        // pos == T: the tail (w < g) into the next slot 0, whose
                        // own cells the next pair writes (after the last pair:
                        // the chain's extra slot, zero there)
                        if (ww < g) *o = v;
                        else if (p.last) *o = 0.f;
                    }
                }
        }
    }
}

// ---- the sweep ----------------------------------------------------------------
template <int NG>
__device__ __forceinline__ void vb_fetch(float *dst, const float *src) {
    constexpr int BYTES = NG * 4;
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (BYTES >= 16) {
#pragma unroll
        for (int o = 0; o < BYTES; o += 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + o), "l"((const char *)src + o)
                         : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(src), "n"(BYTES) : "memory");
    }
}
__device__ __forceinline__ void vb_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void vb_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A lane's position in its chain: pair j (j = np: past the last pair), macro-
// step pos of it (negative before the lane enters the chain), the pair's
// macro-step count and the float offset of its slot 0.
struct VbCursor {
    int j, pos, T, nextT;
    int64_t cur;
};

template <int R, int LAM, int MINB>
__global__ void __launch_bounds__(VB_WARPS * 32, MINB) vband_sweep_kernel(VbArgs a, int cls) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int H = R / 2;
    constexpr int NH = NG / 2;
    constexpr int JOUT = R - 2;
    constexpr int SLOT = NG * NG;
    constexpr int64_t PSTR = 32LL * SLOT;   // floats per slot (all lanes)
    static_assert(R % S == 0 && NG % 2 == 0 && NG <= 16, "2 to 16 coarse rows per lane, even");
    extern __shared__ __align__(16) float vring[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const VbClassInfo ci = a.cinfo[cls];
    const int c = blockIdx.x * VB_WARPS + warp;
    if (c >= ci.W) return;   // whole warp
    const int gc = ci.chain0 + c;
    const int off = a.chain_off[gc];
    const int np = a.chain_off[gc + 1] - off;
    const int *cT = a.cT + off;
    const int *cpid = a.cpid + off;
    constexpr int LS = vb_lane_stride(NG);
    float *ring = vring + (size_t)warp * VB_RING * 32 * LS + lane * LS;   // entry e at + e * 32 LS

    // the chain's length in macro-steps, summed across the lanes
    int tsum = 0;
    for (int j = lane; j < np; j += 32) tsum += cT[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(FULL, tsum, o);
    const int total_m = tsum + 32;

    // consumer (the sweep) and fetcher (VB_RING - 1 windows ahead) cursors
    VbCursor cc, fc;
    cc.j = 0;
    cc.pos = -lane;
    cc.T = cT[0];
    cc.nextT = np > 1 ? cT[1] : 1;
    cc.cur = a.chain_base[gc];
    fc = cc;
    int fw = 0;   // window of the fetcher within its macro-step
    auto advance = [&](VbCursor &q) {
        if (++q.pos == q.T && q.j < np) {
            q.pos = 0;
            q.cur += (int64_t)q.T * PSTR;
            ++q.j;
            q.T = q.nextT;
            q.nextT = q.j + 1 < np ? cT[q.j + 1] : 1;
        }
    };
    auto fetch = [&](int e) {
        float *dst = ring + e * 32 * LS;
        const bool live = fc.pos >= 0 && (fc.j < np || (fc.j == np && fc.pos == 0));
        if (live) {
            vb_fetch<NG>(dst, a.band + fc.cur + ((int64_t)fc.pos * 32 + lane) * SLOT + fw * NG);
        } else {
#pragma unroll
            for (int g = 0; g < NG; g += 2) *reinterpret_cast<float2 *>(dst + g) = make_float2(0.f, 0.f);
        }
        vb_commit();
        if (++fw == NG) {
            fw = 0;
            advance(fc);
        }
    };
#pragma unroll
    for (int e = 0; e < VB_RING - 1; ++e) fetch(e);

    float2 KP[H], QP[H];
    float2 CN[NH], CO[NH];
#pragma unroll
    for (int i = 0; i < H; ++i) { KP[i] = make_float2(1.f, 1.f); QP[i] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int g = 0; g < NH; ++g) { CN[g] = make_float2(0.f, 0.f); CO[g] = CN[g]; }
    float pK = 1.f, pQ = 0.f;
    int e = 0;   // ring entry of the current window

    for (int m = 0; m < total_m; ++m) {
        const bool trans = cc.pos == 0;
#pragma unroll
        for (int w = 0; w < NG; ++w) {
            // window u + VB_RING - 1 into the entry window u - 1 used; then
            // window u has landed
            fetch(e == 0 ? VB_RING - 1 : e - 1);
            vb_wait<VB_RING - 1>();
            const float *cw = ring + e * 32 * LS;
#pragma unroll
            for (int g = 0; g < NH; ++g) CO[g] = CN[g];
            if constexpr (NG >= 4) {
#pragma unroll
                for (int h = 0; h < NG / 4; ++h) {   // groups (2h, 2h + NH), (2h + 1, 2h + 1 + NH)
                    const float4 v = *reinterpret_cast<const float4 *>(cw + 4 * h);
                    CN[2 * h] = make_float2(v.x, v.y);
                    CN[2 * h + 1] = make_float2(v.z, v.w);
                }
            } else {
                CN[0] = *reinterpret_cast<const float2 *>(cw);
            }
            e = e + 1 == VB_RING ? 0 : e + 1;
#pragma unroll
            for (int jj = 0; jj < S; ++jj) {
                const int j = w * S + jj;
                const float kH1 = KP[H - 1].x, qH1 = QP[H - 1].x;   // row H-1 before this step
                float shK = 0.f, shQ = 0.f;
#pragma unroll
                for (int i = H - 1; i >= 0; --i) {
                    const int g1 = i / S, s1 = i % S;   // row i; row i+H: group g1+NH, same s1
                    if (jj == s1 && trans) {            // row starts its next pair now: k(.,0) = 1
                        if (g1 == w) KP[i].x = 1.f;
                        if (g1 + NH == w) KP[i].y = 1.f;
                    }
                    const float2 cf = (jj >= s1) ? CN[g1] : CO[g1];
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
                        // row R-1 of lane 31 just finished the previous pair's last column
                        if (j == JOUT && trans && lane == 31 && cc.j >= 1 && cc.j <= np)
                            a.out[a.plan[cpid[cc.j - 1]].out0] = KP[i].y;
                    }
                }
                pK = (lane == 0) ? 1.f : shK;
                pQ = (lane == 0) ? 0.f : shQ;
            }
        }
        advance(cc);
    }
    vb_wait<0>();
}

// Instances: (R, lambda, MINB).  The classes of dyadic order lambda are the
// instances' R in ascending order.
#define SIGK_VBAND_CASES(X)                                                                   \
    X(4, 0, 6) X(8, 0, 6) X(16, 0, 6) X(4, 1, 6) X(8, 1, 6) X(16, 1, 6) X(32, 1, 4) X(8, 2, 6)   \
    X(16, 2, 6) X(32, 2, 4)

template <int R, int LAM>
constexpr int vb_ring_bytes() { return VB_WARPS * VB_RING * 32 * vb_lane_stride(R >> LAM) * 4; }

template <int R, int LAM, int MINB>
int vb_occupancy() {
    int nb = 0;
    auto kern = vband_sweep_kernel<R, LAM, MINB>;
    const int smem = vb_ring_bytes<R, LAM>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, VB_WARPS * 32, smem) != cudaSuccess) return 0;
    return nb;
}

template <int R, int LAM, int MINB>
cudaError_t vb_launch_sweep(const VbArgs &a, int cls, int grid, cudaStream_t st) {
    auto kern = vband_sweep_kernel<R, LAM, MINB>;
    const int smem = vb_ring_bytes<R, LAM>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, VB_WARPS * 32, smem, st>>>(a, cls);
    return cudaGetLastError();
}

// The same slots with a thread on WQ windows x 2 HB groups, the HB group
// pairs (h, h + NG/2) for h = h0 .. h0 + HB - 1: per channel 2 HB of its
// lane's row increments (two 16-byte loads) and WQ + NG/2 + HB - 1 column
// increments (a broadcast) for 2 HB WQ products, half the lane-distinct
// shared-memory reads a product of vb_coef_kernel's NG = 16 instance; and a
// window row's pairs are 2 HB consecutive floats of the slot.
template <int NG, int WQ, int HB>
__global__ void __launch_bounds__(VB_CT) vb_coef_pair_kernel(VbArgs a, int cls, int dc) {
    extern __shared__ __align__(16) float vcs[];
    constexpr int NPP = 32 * NG, XL = vb_lane_stride(NG), XS = vb_xstride<NG>(), SLOT = NG * NG;
    constexpr int NH = NG / 2, NHB = NH / HB, NQW = NG / WQ;
    constexpr int YN = WQ + NH + HB - 1, YL = (YN + 3) / 4 * 4;
    static_assert(NH % HB == 0 && HB % 4 == 0 && WQ % 4 == 0 && (NH - HB) % 4 == 0, "aligned vector loads");
    const VbClassInfo ci = a.cinfo[cls];
    const int64_t d = a.src.d;
    float *dxs = vcs;
    float *dys = vcs + dc * XS;
    for (int t = blockIdx.x; t < ci.count; t += gridDim.x) {
        const int pid = a.order[ci.start + t];
        const VbPair p = a.plan[pid];
        const float *rows = (const float *)(p.swapped ? a.src.B : a.src.A) + p.r_row0 * d;
        const float *cols = (const float *)(p.swapped ? a.src.A : a.src.B) + p.c_row0 * d;
        const int nx = p.lr - 1, ny = p.lc - 1, T = p.T, NQ = T * NG;
        const int YS = vb_ystride(T, NG);
        const int nthr = 32 * (T + 1) * NQW * NHB;
        for (int b0 = 0; b0 < nthr; b0 += VB_CT) {
            const int u = b0 + (int)threadIdx.x;
            const int l = u & 31, pq = u >> 5;
            const int hb = pq % NHB, pq2 = pq / NHB;
            const int pos = pq2 / NQW, w0 = (pq2 - pos * NQW) * WQ, h0 = hb * HB;
            float acc[WQ][2 * HB];   // [w][2k]: group h0 + k, [w][2k + 1]: group h0 + k + NH
#pragma unroll
            for (int w = 0; w < WQ; ++w)
#pragma unroll
                for (int k = 0; k < 2 * HB; ++k) acc[w][k] = 0.f;
            for (int64_t c0 = 0; c0 < d; c0 += dc) {
                if (d > dc || b0 == 0) {
                    __syncthreads();
                    const int dq = dc / 4;
                    for (int v = threadIdx.x; v < dq * NPP; v += VB_CT) {
                        const int P = v / dq, c = 4 * (v - (v / dq) * dq);
                        const int pr = P - p.vrows;
                        float e[4] = {0.f, 0.f, 0.f, 0.f};
                        if (pr >= 0 && pr < nx) vb_inc4(e, rows + (int64_t)pr * d, d, c0 + c);
                        float *o = dxs + c * XS + (P / NG) * XL + P % NG;
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[k * XS] = e[k];
                    }
                    for (int v = threadIdx.x; v < dq * YS; v += VB_CT) {
                        const int iq = v / dq, c = 4 * (v - (v / dq) * dq);
                        const int q = iq - (NG - 1) - p.nqv;   // real column
                        float e[4] = {0.f, 0.f, 0.f, 0.f};
                        if (q >= 0 && q < ny && iq - (NG - 1) < NQ) vb_inc4(e, cols + (int64_t)q * d, d, c0 + c);
                        float *o = dys + c * YS + iq;
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[k * YS] = e[k];
                    }
                    __syncthreads();
                }
                if (u < nthr) {
                    const int cn = (int)(d - c0 < dc ? d - c0 : dc);
#pragma unroll 2
                    for (int c = 0; c < cn; ++c) {
                        float xa[HB], xb[HB], yv[YL];
                        vb_lds<HB>(xa, dxs + c * XS + l * XL + h0);
                        vb_lds<HB>(xb, dxs + c * XS + l * XL + h0 + NH);
                        // column index Q + NG - 1 = pos NG + w - g, from jb = w0 - h0 + NH - HB
                        vb_lds<YL>(yv, dys + c * YS + pos * NG + w0 - h0 + NH - HB);
#pragma unroll
                        for (int w = 0; w < WQ; ++w)
#pragma unroll
                            for (int k = 0; k < HB; ++k) {
                                acc[w][2 * k] = fmaf(xa[k], yv[w - k + NH - 1 + HB], acc[w][2 * k]);
                                acc[w][2 * k + 1] = fmaf(xb[k], yv[w - k + HB - 1], acc[w][2 * k + 1]);
                            }
                    }
                }
            }
            if (u >= nthr) continue;
#pragma unroll
            for (int w = 0; w < WQ; ++w)
#pragma unroll
                for (int k = 0; k < 2 * HB; ++k) acc[w][k] = scheme_coef(acc[w][k] * a.scale, a.src.scheme);
            float *dst = a.band + p.base + ((int64_t)pos * 32 + l) * SLOT;   // pos = T: the next slot 0
            if (pos > 0 && pos < T) {
#pragma unroll
                for (int w = 0; w < WQ; ++w)
#pragma unroll
                    for (int k = 0; k < 2 * HB; k += 4)
                        *reinterpret_cast<float4 *>(dst + (w0 + w) * NG + 2 * h0 + k) =
                            make_float4(acc[w][k], acc[w][k + 1], acc[w][k + 2], acc[w][k + 3]);
                continue;
            }
#pragma unroll
            for (int w = 0; w < WQ; ++w)
#pragma unroll
                for (int k = 0; k < 2 * HB; ++k) {
                    const int g = (k & 1) ? h0 + (k >> 1) + NH : h0 + (k >> 1);
                    const int ww = w0 + w;
                    float *o = dst + ww * NG + 2 * h0 + k;   // vb_gpos(g)
                    if (pos == 0) {
                        if (ww >= g) *o = acc[w][k];
                        else if (p.first) *o = 0.f;
                    } else {
                        if (ww < g) *o = acc[w][k];
                        else if (p.last) *o = 0.f;
                    }
                }
        }
    }
}

template <int NG, int WQ, int HB>
cudaError_t vb_launch_coef_pair(const VbArgs &a, int cls, int dc, int tmax, int sms, cudaStream_t st) {
    auto kern = vb_coef_pair_kernel<NG, WQ, HB>;
    const int smem = (int)sizeof(float) * dc * (vb_xstride<NG>() + vb_ystride(tmax, NG));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VB_CT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<sms * per_sm, VB_CT, smem, st>>>(a, cls, dc);
    return cudaGetLastError();
}

template <int NG, int WQ>
cudaError_t vb_launch_coef(const VbArgs &a, int cls, int dc, int tmax, int sms, cudaStream_t st) {
    auto kern = vb_coef_kernel<NG, WQ>;
    const int smem = (int)sizeof(float) * dc * (vb_xstride<NG>() + vb_ystride(tmax, NG));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VB_CT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<sms * per_sm, VB_CT, smem, st>>>(a, cls, dc);
    return cudaGetLastError();
}

cudaError_t vb_coef_of(const VbArgs &a, int cls, int NG, int dc, int tmax, int sms, cudaStream_t st) {
    switch (NG) {
        case 2: return vb_launch_coef<2, 2>(a, cls, dc, tmax, sms, st);
        case 4: return vb_launch_coef<4, 4>(a, cls, dc, tmax, sms, st);
        case 8: return vb_launch_coef<8, 8>(a, cls, dc, tmax, sms, st);
        case 16: return vb_launch_coef_pair<16, 8, 4>(a, cls, dc, tmax, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

// The classes of dyadic order lam (ascending R).
int vb_classes(int lam, int *R) {
    int n = 0;
#define X(r, l, mb) if (l == lam && n < VB_NCLS) R[n++] = r;
    SIGK_VBAND_CASES(X)
#undef X
    return n;
}

// Upper bound of T over pairs with paths of at most max_len points.
int vb_tmax(int lam, int64_t max_len, int Rmin) {
    const int64_t Nj = (max_len - 1) << lam;
    const int64_t t = (Nj + Rmin - 1) / Rmin;
    return (int)(t < 2 ? 2 : t);
}

struct VbLayout {
    int64_t plan, order, hist, cinfo, chain_base, chain_off, cpid, cT, scan, band, total;
};

int64_t up256(int64_t v) { return (v + 255) / 256 * 256; }

VbLayout vb_layout(int64_t n, int64_t max_len, int lam) {
    int R[VB_NCLS];
    const int nc = vb_classes(lam, R);
    const int S = 1 << lam;
    const int TK = vb_tmax(lam, max_len, R[0]) + 1;
    VbLayout L;
    int64_t o = 256;   // a 256-byte header: the status word that sigk_stream_status reads (no waits here: 0)
    L.plan = o; o = up256(o + n * (int64_t)sizeof(VbPair));
    L.order = o; o = up256(o + n * 4);
    L.hist = o; o = up256(o + (int64_t)nc * TK * 4);
    L.cinfo = o; o = up256(o + VB_NCLS * (int64_t)sizeof(VbClassInfo));
    L.chain_base = o; o = up256(o + n * 8);
    L.chain_off = o; o = up256(o + (n + 1) * 4);
    L.cpid = o; o = up256(o + n * 4);
    L.cT = o; o = up256(o + n * 4);
    L.scan = o; o = up256(o + n * 8);
    // band: a pair of class R takes (T + 1) slots of 32 (R / S)^2 floats at
    // most (its slots and, as a chain's last pair, the extra slot); the bound
    // takes the largest over the classes of the longest pair
    int64_t per = 0;
    for (int c = 0; c < nc; ++c) {
        const int64_t ng = R[c] / S;
        const int64_t t = vb_tmax(lam, max_len, R[c]);
        const int64_t f = (t + 1) * 32 * ng * ng;
        if (f > per) per = f;
    }
    L.band = o;
    o = up256(o + n * per * (int64_t)sizeof(float));
    L.total = o;
    return L;
}

// The classes' contractions and sweeps are independent: they run on streams
// of their own, forked from and joined back to the caller's stream by events
// (which a stream capture records as a forked graph).  Created once per
// device, on first use.
struct VbStreams {
    bool ok;
    cudaStream_t s[VB_NCLS];
    cudaEvent_t fork, join[VB_NCLS];
};
constexpr int VB_MAX_DEVICES = 64;
std::mutex g_vb_mu;
VbStreams g_vb[VB_MAX_DEVICES];

cudaError_t vb_streams(int dev, VbStreams **out) {
    if (dev < 0 || dev >= VB_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_vb_mu);
    VbStreams &v = g_vb[dev];
    if (!v.ok) {
        cudaError_t e = cudaEventCreateWithFlags(&v.fork, cudaEventDisableTiming);
        for (int c = 0; c < VB_NCLS && e == cudaSuccess; ++c) {
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

bool vband_supported(int lam, int64_t d, int64_t max_len, int dtype, int kernel) {
    if (dtype != SIGK_F32 || kernel != SIGK_KERNEL_LINEAR || d < 1 || max_len < 1) return false;
    int R[VB_NCLS];
    const int nc = vb_classes(lam, R);
    if (nc == 0) return false;
    return ((max_len - 1) << lam) <= 32LL * R[nc - 1];
}

int64_t vband_workspace_bytes(int64_t n, int64_t max_len, int lam) {
    return n <= 0 ? 0 : vb_layout(n, max_len, lam).total;
}

cudaError_t launch_vband(const PairSrc &src, int64_t n, int lam, int64_t max_len, float *out, void *ws,
                         cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const VbLayout L = vb_layout(n, max_len, lam);
    unsigned char *w = (unsigned char *)ws;
    VbArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.out = out;
    a.band = (float *)(w + L.band);
    a.plan = (VbPair *)(w + L.plan);
    a.order = (int *)(w + L.order);
    a.hist = (int *)(w + L.hist);
    a.cinfo = (VbClassInfo *)(w + L.cinfo);
    a.chain_base = (int64_t *)(w + L.chain_base);
    a.chain_off = (int *)(w + L.chain_off);
    a.cpid = (int *)(w + L.cpid);
    a.cT = (int *)(w + L.cT);
    a.scan = (int64_t *)(w + L.scan);
    a.n = n;
    a.lam = lam;
    a.ncls = vb_classes(lam, a.R);
    a.TK = vb_tmax(lam, max_len, a.R[0]) + 1;
    a.scale = 0.5f / (float)(1 << (2 * lam));
    for (int c = 0; c < a.ncls; ++c) {
        int occ = 0;
#define X(r, l, mb) if (r == a.R[c] && l == lam) occ = vb_occupancy<r, l, mb>();
        SIGK_VBAND_CASES(X)
#undef X
        if (occ < 1) return cudaErrorInvalidConfiguration;
        a.cap[c] = sms * occ * VB_WARPS;
    }
    if ((e = cudaMemsetAsync(w, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.hist, 0, (size_t)a.ncls * a.TK * 4, st)) != cudaSuccess) return e;
    const int pgrid = (int)((n + 255) / 256 < (int64_t)sms * 4 ? (n + 255) / 256 : (int64_t)sms * 4);
    vb_pairs_kernel<<<pgrid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    vb_plan_kernel<<<1, VB_PT, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int dc = (int)(src.d < VB_DC ? ((src.d + 3) / 4) * 4 : VB_DC);
    VbStreams *vs = nullptr;
    if ((e = vb_streams(dev, &vs)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(vs->fork, st)) != cudaSuccess) return e;
    for (int c = 0; c < a.ncls; ++c) {
        cudaStream_t sc = vs->s[c];
        if ((e = cudaStreamWaitEvent(sc, vs->fork, 0)) != cudaSuccess) return e;
        const int ng = a.R[c] >> lam;
        if ((e = vb_coef_of(a, c, ng, dc, vb_tmax(lam, max_len, a.R[c]), sms, sc)) != cudaSuccess) return e;
        const int grid = (a.cap[c] + VB_WARPS - 1) / VB_WARPS;
        bool launched = false;
#define X(r, l, mb)                                                          \
        if (r == a.R[c] && l == lam) {                                       \
            if ((e = vb_launch_sweep<r, l, mb>(a, c, grid, sc)) != cudaSuccess) return e; \
            launched = true;                                                 \
        }
        SIGK_VBAND_CASES(X)
#undef X
        if (!launched) return cudaErrorInvalidValue;
        if ((e = cudaEventRecord(vs->join[c], sc)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, vs->join[c], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sigk
