// Forward sweep for long or uneven pairs: the grid of each pair is cut into
// horizontal strips of 32*R refined rows; a persistent kernel hands strips to
// warps in pair order from an atomic counter, and the strips of one pair form
// a wavefront across warps (Sec. 3.1.1's anti-diagonal parallelism carried
// from one warp to the next): each strip writes its bottom row column by
// column into a buffer that the strip below reads in chunks of CW columns.
// The buffer is filled with an all-ones bit pattern before the sweep, a NaN
// that no arithmetic result has, so a value carries its own readiness: the
// writer uses relaxed stores with no flag and no fence, and the reader loads a
// chunk with relaxed loads half a chunk before it needs it and polls again
// only where some lane still sees the pattern.
//
// Inside a strip the work is laid out as in the chained kernel: lane l holds
// rows R*l .. R*l+R-1, row r of lane l works on column t - R*l - r + 1 at step
// t, and the scheme runs in its difference form
//   Q(a,b) = Q(a-1,b) + c (K(a,b-1) + K(a-1,b)),  K(a,b) = K(a,b-1) + Q(a,b),
// c = 1/2 4^-lambda <dx_p, dy_q> (Sec. 3.1, scheme and remark).
//
// Coefficients: a separate kernel forms every coarse-cell coefficient c(p,q)
// once and stores each strip's coefficients anti-diagonal-major, d(n, P) =
// c(p, n - P) for the strip's coarse rows P: at window n every group of every
// lane of the warp needs exactly diagonal n (the skew of the wavefront makes
// p + q the same for all of them), so a lane reads its NG coefficients as
// contiguous vectors and the warp reads one contiguous slice.  Virtual rows
// (above a pair's first row, padding the first strip) and columns outside the
// grid have c = 0, which keeps K = 1 and Q = 0 exactly there.
//
// Waits are bounded: a reader that does not see its chunk within
// `wait_cycles` records SIGK_ETIMEOUT in the status word and carries on
// (its result is then meaningless and the call reports the timeout).
#include <string.h>

#include <type_traits>

#include "rbf.cuh"
#include "sigk_internal.cuh"
#include "tc5.cuh"

namespace sigk {

namespace {

constexpr int STRIP_WARPS = 2;   // warps per CTA
constexpr int CW = 32;           // columns per published chunk of a bottom row

// Steps between the backward's checkpoints of the forward state: the adjoint
// undoes the steps in between in place, and each undo rounds once more.
template <typename T>
__host__ __device__ constexpr int strip_ck() { return sizeof(T) == 4 ? 64 : 128; }
inline int strip_ck_of(int64_t es) { return es == 4 ? 64 : 128; }

// ---- planning: per-pair sizes and offsets, computed on the device ----------

struct PairPlan {
    int64_t a_row0, b_row0;  // first point row of the row path and column path
    int64_t c_off;           // start of this pair's coefficient blocks (elements)
    int64_t bnd_off;         // start of its bottom-row buffers (elements)
    int64_t strip_base;      // global index of its first strip
    int64_t out0, out1;
    int ni, nj;              // refined rows / columns
    int nx, ny;              // coarse rows / columns
    int ns, pad;             // strips, virtual refined rows above the first
    int nw;                  // windows (coefficient diagonals) per strip
    int swap;                // 1: the rows refine the B path (src.B), columns the A path
    int64_t s_off;           // backward: start of its checkpoints of the forward state
    int64_t g_off;           // backward: start of its dense dk/dG [nx][ny]
};

// totals[]: the sums of the coefficient, boundary-row, strip, sums and dk/dG
// sizes over all pairs
constexpr int TOT_STRIPS = 2;

// ck: steps between the backward's checkpoints (0: forward only); with it
// every strip, the last too, keeps its bottom row
template <int R, int LAM>
__global__ void plan_kernel(PairSrc src, int64_t n, PairPlan *plan, int64_t *totals, int shorter_rows,
                            int ck) {
    constexpr int S = 1 << LAM;
    constexpr int TH = 32 * R;
    constexpr int CP = 32 * (R / S);
    __shared__ int64_t part[5][512];
    // pass 1: per-pair shape
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const PairRef pr = pair_ref(src, k);
        PairPlan p;
        // rows refine the longer path (more strips, more warps per pair) or,
        // with many pairs in flight, the shorter one (fewer virtual rows and
        // fill/drain steps per cell)
        const bool swap = shorter_rows ? pr.la > pr.lb : pr.lb > pr.la;
        const int64_t la = swap ? pr.lb : pr.la, lb = swap ? pr.la : pr.lb;
        p.a_row0 = swap ? pr.b_row0 : pr.a_row0;
        p.b_row0 = swap ? pr.a_row0 : pr.b_row0;
        p.out0 = pr.out0;
        p.out1 = pr.out1;
        p.swap = swap ? 1 : 0;
        p.nx = la > 1 ? (int)(la - 1) : 0;
        p.ny = lb > 1 ? (int)(lb - 1) : 0;
        p.ni = p.nx << LAM;
        p.nj = p.ny << LAM;
        p.ns = (p.nx > 0 && p.ny > 0) ? (p.ni + TH - 1) / TH : 0;
        p.pad = p.ns * TH - p.ni;
        p.nw = ((p.nj + TH - 2) >> LAM) + 2;
        p.c_off = (int64_t)p.ns * p.nw * CP;        // sizes for now, offsets after the scan
        p.bnd_off = p.ns > 0 ? (int64_t)(ck ? p.ns : p.ns - 1) * p.nj * 2 : 0;
        p.strip_base = p.ns;
        p.s_off = ck ? (int64_t)p.ns * ((p.nj + TH - 1 + ck - 1) / ck) * TH * 2 : 0;
        p.g_off = (int64_t)p.nx * p.ny;
        plan[k] = p;
    }
    __syncthreads();
    // pass 2: exclusive scans of the five sizes, in chunks of blockDim
    int64_t run[5] = {0, 0, 0, 0, 0};
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        int64_t v[5] = {0, 0, 0, 0, 0};
        if (k < n) {
            v[0] = plan[k].c_off;
            v[1] = plan[k].bnd_off;
            v[2] = plan[k].strip_base;
            v[3] = plan[k].s_off;
            v[4] = plan[k].g_off;
        }
        for (int j = 0; j < 5; ++j) part[j][threadIdx.x] = v[j];
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int64_t t[5];
            for (int j = 0; j < 5; ++j)
                t[j] = (int)threadIdx.x >= off ? part[j][threadIdx.x - off] : 0;
            __syncthreads();
            for (int j = 0; j < 5; ++j) part[j][threadIdx.x] += t[j];
            __syncthreads();
        }
        if (k < n) {
            plan[k].c_off = run[0] + part[0][threadIdx.x] - v[0];
            plan[k].bnd_off = run[1] + part[1][threadIdx.x] - v[1];
            plan[k].strip_base = run[2] + part[2][threadIdx.x] - v[2];
            plan[k].s_off = run[3] + part[3][threadIdx.x] - v[3];
            plan[k].g_off = run[4] + part[4][threadIdx.x] - v[4];
        }
        for (int j = 0; j < 5; ++j) run[j] += part[j][blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < 5; ++j) totals[j] = run[j];
}

// ---- increments: dx_r = x_{r+1} - x_r for every point row r of a path array,
// stored at row r (the last row of each path is never read), channels padded
// to a multiple of 4 with zeros so that a row is a run of 16-byte vectors.

template <typename T>
__global__ void inc_kernel(const T *pts, int64_t rows, const int64_t *rows_dev, int64_t d,
                           int64_t D4, T *inc) {
    // rows_dev: the exact row count of a packed array (its last offset), when
    // the host only knows an upper bound
    if (rows_dev && *rows_dev < rows) rows = *rows_dev;
    const int64_t total = rows * D4 * 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / (D4 * 4), c = i - (i / (D4 * 4)) * (D4 * 4);
        inc[i] = (c < d && r + 1 < rows) ? pts[(r + 1) * d + c] - pts[r * d + c] : (T)0;
    }
}

// ---- coefficients: each strip's anti-diagonal-major block -----------------
// One CTA computes 64 diagonals x 64 strip rows at a time; thread (tx, ty)
// computes rows P0 + tx + 16 j and diagonals W0 + ty + 16 i (i, j < 4): its
// 16 outputs need 4 row-path and 7 column-path increment vectors (the column
// q = W - P depends on i - j only), read from shared memory as 4-channel
// vectors; adjacent threads read adjacent rows, which an odd row stride keeps
// free of bank conflicts, and store adjacent outputs.

constexpr int GT = 64;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> { using type = float4; };
template <>
struct Vec4<double> { using type = double4_32a; };

template <typename T, int R, int LAM>
__global__ void __launch_bounds__(256) coef_kernel(PairSrc src, const PairPlan *plan,
                                                   int64_t n_pairs, const int64_t *totals,
                                                   const T *incA, const T *incB, T *cbuf) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int CP = 32 * NG;      // coarse rows per strip (incl. virtual)
    using V4 = typename Vec4<T>::type;
    extern __shared__ unsigned char smraw[];
    const int64_t d = src.d;
    const int D4 = (int)((d + 3) / 4);
    const int RS = D4 | 1;   // odd row stride in V4 units: conflict-free row-adjacent reads
    V4 *sx = reinterpret_cast<V4 *>(smraw);          // GT rows of dx
    V4 *sy = sx + GT * RS;                            // 2*GT-1 rows of dy
    const T scale = (T)0.5 / (T)(1LL << (2 * LAM));
    const int64_t total_strips = totals[TOT_STRIPS];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int64_t gs = blockIdx.x; gs < total_strips; gs += gridDim.x) {
        // the pair of this strip: last plan with strip_base <= gs
        int64_t lo = 0, hi = n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (plan[mid].strip_base <= gs) lo = mid; else hi = mid - 1;
        }
        const PairPlan pp = plan[lo];
        const int s = (int)(gs - pp.strip_base);
        // a_row0 / b_row0 are offsets into the row / column path's own array
        const V4 *x = reinterpret_cast<const V4 *>(pp.swap ? incB : incA) + pp.a_row0 * D4;
        const V4 *y = reinterpret_cast<const V4 *>(pp.swap ? incA : incB) + pp.b_row0 * D4;
        T *blk = cbuf + pp.c_off + (int64_t)s * pp.nw * CP;
        const int prow0 = s * CP - (pp.pad >> LAM);   // real coarse row of strip row 0
        for (int W0 = 0; W0 < pp.nw; W0 += GT) {
            for (int P0 = 0; P0 < CP; P0 += GT) {
                // a tile whose rows are all virtual or whose columns q = W - P all
                // fall outside the grid holds zeros only
                const int plo = prow0 + P0 > 0 ? prow0 + P0 : 0;
                const int phi = prow0 + P0 + GT - 1 < pp.nx - 1 ? prow0 + P0 + GT - 1 : pp.nx - 1;
                const int qlo = W0 - (P0 + GT - 1), qhi = W0 + GT - 1 - P0;
                if (plo > phi || qhi < 0 || qlo >= pp.ny) {
                    for (int u = threadIdx.x; u < GT * GT; u += blockDim.x) {
                        const int W = W0 + u / GT, P = P0 + (u % GT);
                        if (W < pp.nw && P < CP) blk[(int64_t)W * CP + P] = (T)0;
                    }
                    continue;
                }
                __syncthreads();
                // stage dx rows P0 .. P0+GT-1 and dy rows q = W - P in [W0-P0-GT+1, W0-P0+GT-1]
                for (int u = threadIdx.x; u < GT * D4; u += blockDim.x) {
                    const int i = u / D4, c4 = u - (u / D4) * D4;
                    const int p = prow0 + P0 + i;
                    V4 w;
                    if (p >= 0 && p < pp.nx) w = x[(int64_t)p * D4 + c4];
                    else { w.x = 0; w.y = 0; w.z = 0; w.w = 0; }
                    sx[i * RS + c4] = w;
                }
                const int q0 = W0 - P0 - (GT - 1);
                for (int u = threadIdx.x; u < (2 * GT - 1) * D4; u += blockDim.x) {
                    const int i = u / D4, c4 = u - (u / D4) * D4;
                    const int q = q0 + i;
                    V4 w;
                    if (q >= 0 && q < pp.ny) w = y[(int64_t)q * D4 + c4];
                    else { w.x = 0; w.y = 0; w.z = 0; w.w = 0; }
                    sy[i * RS + c4] = w;
                }
                __syncthreads();
                // thread (tx, ty): rows P0 + tx + 16 j, diagonals W0 + ty + 16 i
                T acc[4][4];
                for (int i = 0; i < 4; ++i)
                    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
                for (int c4 = 0; c4 < D4; ++c4) {
                    V4 xv[4], yv[7];
#pragma unroll
                    for (int j = 0; j < 4; ++j) xv[j] = sx[(tx + 16 * j) * RS + c4];
#pragma unroll
                    for (int m = 0; m < 7; ++m) {
                        // q - q0 = (ty + 16 i) - (tx + 16 j) + GT - 1, with i - j = m - 3
                        yv[m] = sy[(ty - tx + 16 * (m - 3) + (GT - 1)) * RS + c4];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const V4 a = xv[j], b = yv[i - j + 3];
                            T t = acc[i][j];
                            t = fma(a.x, b.x, t);
                            t = fma(a.y, b.y, t);
                            t = fma(a.z, b.z, t);
                            t = fma(a.w, b.w, t);
                            acc[i][j] = t;
                        }
                }
                for (int i = 0; i < 4; ++i) {
                    const int W = W0 + ty + 16 * i;
                    if (W >= pp.nw) continue;
                    for (int j = 0; j < 4; ++j) {
                        const int P = P0 + tx + 16 * j;
                        if (P >= CP) continue;
                        const int p = prow0 + P, q = W - P;
                        const bool ok = p >= 0 && p < pp.nx && q >= 0 && q < pp.ny;
                        blk[(int64_t)W * CP + P] = ok ? scheme_coef(acc[i][j] * scale, src.scheme) : (T)0;
                    }
                }
            }
        }
    }
}

// ---- the persistent strip sweep --------------------------------------------

// The strip boundary rows: relaxed accesses at GPU scope, each value read or
// written whole; the all-ones pattern marks a value not yet written.
__device__ __forceinline__ float ld_relaxed(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_relaxed(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ bool unwritten(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ bool unwritten(double v) { return __double_as_longlong(v) == -1LL; }
// a value that happens to have the pattern (only a NaN can) is stored as
// another NaN: the unsigned minimum with all-ones-but-one leaves every other
// bit pattern as it is
__device__ __forceinline__ void st_boundary(float *p, float v) {
    const unsigned b = umin(__float_as_uint(v), 0xfffffffeu);
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(b));
}
__device__ __forceinline__ void st_boundary(double *p, double v) {
    const unsigned long long b = ullmin((unsigned long long)__double_as_longlong(v), 0xfffffffffffffffeULL);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b));
}
// the same store under a predicate, without a branch around it
__device__ __forceinline__ void st_boundary_if(float *p, float v, bool pred) {
    const unsigned b = umin(__float_as_uint(v), 0xfffffffeu);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.relaxed.gpu.global.b32 [%0], %1;\n\t}"
                 ::"l"(p), "r"(b), "r"((int)pred));
}
__device__ __forceinline__ void st_boundary_if(double *p, double v, bool pred) {
    const unsigned long long b = ullmin((unsigned long long)__double_as_longlong(v), 0xfffffffffffffffeULL);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.relaxed.gpu.global.b64 [%0], %1;\n\t}"
                 ::"l"(p), "l"(b), "r"((int)pred));
}

template <typename T>
struct StripArgs {
    PairSrc src;
    const PairPlan *plan;
    const int64_t *totals;
    int64_t n_pairs;
    const T *cbuf;
    T *bnd;          // boundary rows, filled with the all-ones pattern first
    int *counter;
    int *status;
    T *out;
    long long wait_cycles;
    int fault_inject;   // 1: the first strip of the first pair never publishes
    T *sums;            // backward: checkpoints of the state, [strip][step / ck][lane][K 0..R-1, Q 0..R-1]
};

constexpr int NRING = 8;   // coefficient diagonals in flight per warp

// Each lane copies its own NG coefficients of a diagonal into the warp's ring
// (cp.async, so the copy needs no registers), NRING - 1 diagonals ahead.
template <typename T, int NG>
__device__ __forceinline__ void ring_fetch(T *slot, const T *src) {
    constexpr int BYTES = NG * (int)sizeof(T);
    constexpr int CH = BYTES >= 16 ? 16 : BYTES;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(slot);
#pragma unroll
    for (int o = 0; o < BYTES; o += CH) {
        if (CH == 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + o),
                         "l"((const char *)src + o) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst + o),
                         "l"((const char *)src + o), "n"(CH) : "memory");
    }
}

__device__ __forceinline__ void ring_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ring_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// SAVE: also keep what the adjoint needs to run the sweep backwards: every
// strip's bottom row (the last strip's too) and, after every ck-th step (and
// the last), the (K, Q) of all the strip's rows (a.sums)
template <typename T, int R, int LAM, bool SAVE>
__global__ void __launch_bounds__(STRIP_WARPS * 32) strip_kernel(StripArgs<T> a) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int CP = 32 * NG;
    constexpr int TH = 32 * R;
    static_assert(R % S == 0, "whole coarse rows per lane");
    __shared__ __align__(16) T topbuf[STRIP_WARPS][CW * 2];
    __shared__ __align__(16) T ring[STRIP_WARPS][NRING][CP];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T *tb = topbuf[warp];
    const int64_t total_strips = a.totals[TOT_STRIPS];

    for (;;) {
        int64_t gs = 0;
        if (lane == 0) gs = atomicAdd((unsigned long long *)a.counter, 1ULL);
        gs = __shfl_sync(FULL, gs, 0);
        if (gs >= total_strips) break;
        int64_t lo = 0, hi = a.n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (a.plan[mid].strip_base <= gs) lo = mid; else hi = mid - 1;
        }
        const PairPlan pp = a.plan[lo];
        const int s = (int)(gs - pp.strip_base);
        const int nj = pp.nj;
        const T *blk = a.cbuf + pp.c_off + (int64_t)s * pp.nw * CP;
        const T *top = s > 0 ? a.bnd + pp.bnd_off + (int64_t)(s - 1) * nj * 2 : nullptr;
        T *bot = (s < pp.ns - 1 || SAVE) ? a.bnd + pp.bnd_off + (int64_t)s * nj * 2 : nullptr;
        const bool mute = a.fault_inject && lo == 0 && s == 0;
        const int tend = nj + TH - 1;   // steps until the last row leaves column nj

        // FP32: rows (i, i + H) and groups (g, g + NH) of a lane in float2s
        // (FADD2/FFMA2: one issue slot for two rows, bit for bit the scalar
        // arithmetic; NG is even for every FP32 instance).  FP64: scalar rows.
        constexpr bool PACK = sizeof(T) == 4;
        constexpr int H = R / 2, NH = NG / 2;
        static_assert(!PACK || NG % 2 == 0, "an even number of coarse rows per lane");
        T K[R], Q[R], cn[NG], co[NG];
        float2 KP[H], QP[H], CN[NH > 0 ? NH : 1], CO[NH > 0 ? NH : 1];
        if constexpr (PACK) {
#pragma unroll
            for (int i = 0; i < H; ++i) { KP[i] = make_float2(1.f, 1.f); QP[i] = make_float2(0.f, 0.f); }
#pragma unroll
            for (int g = 0; g < NH; ++g) { CN[g] = make_float2(0.f, 0.f); CO[g] = CN[g]; }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) { K[r] = 1; Q[r] = 0; }
#pragma unroll
            for (int g = 0; g < NG; ++g) { cn[g] = 0; co[g] = 0; }
        }
        T pK = 1, pQ = 0;
        bool timed_out = false;
        // the top row's chunk c, columns c CW .. c CW + CW - 1, two values a
        // lane: loaded half a chunk before it is published to the warp, and
        // loaded again, within the wait bound, while some lane still sees the
        // unwritten pattern
        T tn0 = 0, tn1 = 0;
        auto load_top = [&](int c) {
            const int col = c * CW + lane;
            tn0 = col < nj ? ld_relaxed(top + (int64_t)col * 2) : (T)0;
            tn1 = col < nj ? ld_relaxed(top + (int64_t)col * 2 + 1) : (T)0;
        };
        auto wait_top = [&](int c) {
            const long long t0 = clock64();
            while (!timed_out && __any_sync(FULL, unwritten(tn0) || unwritten(tn1))) {
                if (__any_sync(FULL, clock64() - t0 > a.wait_cycles)) {
                    timed_out = true;
                    if (lane == 0) atomicExch(a.status, (int)SIGK_ETIMEOUT);
                    break;
                }
                __nanosleep(100);
                load_top(c);
            }
        };
        if (top) {
            // start once chunks 0 and 1 are written: from then on a chunk
            // loaded half a chunk early is there already (both strips step
            // at the same pace)
            load_top(0);
            wait_top(0);
            tb[2 * lane] = tn0;
            tb[2 * lane + 1] = tn1;
            __syncwarp();
            if (CW < nj) {
                load_top(1);
                wait_top(1);
            }
        }
        // fill the ring with diagonals 0 .. NRING-2 (one commit group each)
#pragma unroll
        for (int k = 0; k < NRING - 1; ++k) {
            if (k < pp.nw) ring_fetch<T, NG>(&ring[warp][k][lane * NG], blk + (int64_t)k * CP + lane * NG);
            ring_commit();
        }

        // lane 0 of a strip with a top row takes its row-0 neighbour from the
        // published chunk (columns past nj keep the last); lane 0 of a first
        // strip keeps the boundary K = 1, Q = 0; the other lanes take lane - 1's
        // last row
        const bool top0 = top != nullptr && lane == 0;
        const bool bst = bot != nullptr && !mute && lane == 31;
        constexpr int WPC = CW / S;   // windows per chunk of the top row
        static_assert(WPC >= 2 && CW % (2 * S) == 0, "a chunk spans whole windows, half a chunk too");
        const int nwin = (tend + S - 1) / S;
        const int nfull = tend / S;   // windows whose S steps all lie before tend
        // the next window's coefficients, read from the ring one window ahead
        // so that no step waits on a shared-memory load (diagonal nwin exists:
        // nw >= nwin + 1)
        float2 CX[NH > 0 ? NH : 1];
        T cx[NG];
        auto read_next = [&](int wn) {
            const T *cw = &ring[warp][wn % NRING][lane * NG];
            if constexpr (PACK) {
#pragma unroll
                for (int g = 0; g < NH; ++g) CX[g] = make_float2(cw[g], cw[g + NH]);
            } else {
#pragma unroll
                for (int g = 0; g < NG; ++g) cx[g] = cw[g];
            }
        };
        ring_wait<NRING - 2>();   // diagonal 0 has landed
        read_next(0);
        int tev = top ? WPC : 0x7fffffff;   // the next window with top-row chunk work

        // one window: S steps; TAIL: the last, partial window checks each step
        auto window = [&](int w, auto tail_tag) {
            constexpr bool TAIL = decltype(tail_tag)::value;
            // diagonal w + NRING - 1 into the slot diagonal w - 1 used (read a
            // window ago); then diagonal w + 1 has landed (at most NRING - 2
            // newer groups in flight)
            {
                // past the last diagonal the copy repeats it: slots of
                // diagonals >= nw are never read (nw >= nwin + 1), and an
                // unconditional copy keeps the window free of branches
                const int k = w + NRING - 1;
                const int kc = min(k, pp.nw - 1);
                ring_fetch<T, NG>(&ring[warp][k % NRING][lane * NG], blk + (int64_t)kc * CP + lane * NG);
                ring_commit();
                ring_wait<NRING - 2>();
            }
            if constexpr (PACK) {
#pragma unroll
                for (int g = 0; g < NH; ++g) { CO[g] = CN[g]; CN[g] = CX[g]; }
            } else {
#pragma unroll
                for (int g = 0; g < NG; ++g) { co[g] = cn[g]; cn[g] = cx[g]; }
            }
            read_next(w + 1);
            // the top row at the window's first step t = w S: chunk c = t / CW
            // (columns t+1 .. t+CW) was loaded half a chunk ago, publish it;
            // load chunk c + 1 half a chunk on (chunks 0 and 1 were loaded at
            // the start)
            if (w == tev) {   // warp-uniform: publish or load, every half chunk from window WPC on
                const int c = w / WPC;
                if (w % WPC == 0) {
                    if (c * CW < nj) {
                        wait_top(c);
                        __syncwarp();
                        tb[2 * lane] = tn0;
                        tb[2 * lane + 1] = tn1;
                        __syncwarp();
                    }
                } else if ((c + 1) * CW < nj) {
                    load_top(c + 1);
                }
                tev += WPC / 2;
            }
            // the window's S top-row values (K, Q), read by every lane (one
            // broadcast address) and taken by lane 0 of a strip with a top row
            T topv[2 * S];
            {
                const T *src = tb + ((w * S) % CW) * 2;
#pragma unroll
                for (int e = 0; e < 2 * S; ++e) topv[e] = src[e];
            }
#pragma unroll
            for (int jj = 0; jj < S; ++jj) {
                const int t = w * S + jj;
                if constexpr (TAIL) {
                    if (t >= tend) break;
                }
                // lane 0's row 0 is at column t + 1 now
                if (top0 && t < nj) {
                    pK = topv[2 * jj];
                    pQ = topv[2 * jj + 1];
                }
                T shK = 0, shQ = 0;
                const bool bstore = bst && (unsigned)(t - (TH - 1)) < (unsigned)nj;
                const int bcol = t - (TH - 1);   // zero-based column of the lane's last row
                if constexpr (PACK) {
                    const float kH1 = KP[H - 1].x, qH1 = QP[H - 1].x;   // row H-1 before this step
#pragma unroll
                    for (int i = H - 1; i >= 0; --i) {
                        const int g1 = i / S, s1 = i % S;   // row i; row i+H: group g1+NH, same s1
                        const float2 c = (jj >= s1) ? CN[g1] : CO[g1];
                        float2 ku, qu;
                        if (i > 0) {
                            ku = KP[i > 0 ? i - 1 : 0];
                            qu = QP[i > 0 ? i - 1 : 0];
                        } else {
                            ku = make_float2(pK, kH1);
                            qu = make_float2(pQ, qH1);
                        }
                        const float2 sum = __fadd2_rn(KP[i], ku);
                        const float2 qn = __ffma2_rn(c, sum, qu);
                        KP[i] = __fadd2_rn(KP[i], qn);
                        QP[i] = qn;
                        if (i == H - 1) {
                            shK = __shfl_up_sync(FULL, KP[i].y, 1);
                            shQ = __shfl_up_sync(FULL, QP[i].y, 1);
                            st_boundary_if(bot + (int64_t)bcol * 2, KP[i].y, bstore);
                            st_boundary_if(bot + (int64_t)bcol * 2 + 1, QP[i].y, bstore);
                        }
                    }
                    if constexpr (SAVE) {
                        constexpr int CK = strip_ck<T>();
                        if ((t + 1) % CK == 0 || t == tend - 1) {
                            const int nck = (tend + CK - 1) / CK;
                            T *dst = a.sums + pp.s_off + (((int64_t)s * nck + t / CK) * 32 + lane) * (2 * R);
#pragma unroll
                            for (int i = 0; i < H; ++i) {
                                dst[i] = KP[i].x; dst[i + H] = KP[i].y;
                                dst[R + i] = QP[i].x; dst[R + i + H] = QP[i].y;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int r = R - 1; r >= 0; --r) {
                        const int g = r / S, sr = r % S;
                        const T c = (jj >= sr) ? cn[g] : co[g];
                        const T kl = K[r];
                        const T ku = r > 0 ? K[r > 0 ? r - 1 : 0] : pK;
                        const T qu = r > 0 ? Q[r > 0 ? r - 1 : 0] : pQ;
                        const T sum = kl + ku;
                        const T qn = qu + c * sum;
                        K[r] = kl + qn;
                        Q[r] = qn;
                        if (r == R - 1) {
                            shK = __shfl_up_sync(FULL, K[r], 1);
                            shQ = __shfl_up_sync(FULL, Q[r], 1);
                            st_boundary_if(bot + (int64_t)bcol * 2, K[r], bstore);
                            st_boundary_if(bot + (int64_t)bcol * 2 + 1, Q[r], bstore);
                        }
                    }
                    if constexpr (SAVE) {
                        constexpr int CK = strip_ck<T>();
                        if ((t + 1) % CK == 0 || t == tend - 1) {
                            const int nck = (tend + CK - 1) / CK;
                            T *dst = a.sums + pp.s_off + (((int64_t)s * nck + t / CK) * 32 + lane) * (2 * R);
#pragma unroll
                            for (int r = 0; r < R; ++r) { dst[r] = K[r]; dst[R + r] = Q[r]; }
                        }
                    }
                }
                if (lane != 0) {
                    pK = shK;
                    pQ = shQ;
                }
            }
        };
        // four windows a loop iteration: the loop's own compare and branch
        // cost a step about a tenth of its time at one window an iteration
#pragma unroll 4
        for (int w = 0; w < nfull; ++w) window(w, std::false_type{});
        if (nfull < nwin) window(nfull, std::true_type{});
        ring_wait<0>();
        if (a.out && s == pp.ns - 1 && lane == 31) {
            T kc;
            if constexpr (PACK) kc = KP[H - 1].y; else kc = K[R - 1];
            a.out[pp.out0] = kc;
            if (pp.out1 >= 0) a.out[pp.out1] = kc;
        }
    }
}


// ---- the adjoint: the strip schedule run backwards in time -----------------
// A(a,b) = d k(Ni,Nj) / d K(a,b) obeys (reverse mode of the scheme)
//   P(a,b) = A(a,b) - A(a,b+1) = c(a,b+1) A(a,b+1) + V(a+1,b),
//   V(a,b) = P(a,b) + c(a,b) A(a,b),
// with A(.,Nj+1) = 0 and V(Ni+1,b) = [b = Nj] (the seed A(Ni,Nj) = 1).  Each
// cell needs, from the step after it in the forward schedule, its own A and
// coefficient and the row below's V, so running the forward schedule
// backwards (rows ascending within a step, V passed up the lanes and, between
// strips, through chunked buffers behind bounded waits, strips of a pair in
// reverse order) has every input ready.  Each cell adds A(a,b) (K(a,b-1) +
// K(a-1,b)) to dk/dG of its coarse cell; a group's coarse cell is complete at
// the end of the window whose diagonal it sits on.
//
// The sums K(a,b-1) + K(a-1,b) are not stored: the forward state is run
// backwards with it.  After forward step t row a holds (K(a,b), Q(a,b)) at its
// column b, and the step is undone in place (exact algebra; each undo rounds
// once more in floating point):
//   K(a,b-1) = K(a,b) - Q(a,b),
//   sum      = K(a,b-1) + K(a-1,b)       (the row above's undone K),
//   Q(a,b-1) = Q(a+1,b-1) - c(a+1,b-1) sum(a+1,b-1)   (from the row below).
// The strip's first row takes K(a-1,b) from the strip above's bottom row, its
// last row takes its (K, Q) from its own bottom row (both kept by the
// forward), and the state is reloaded from the forward's checkpoints every ck
// steps, which bounds the drift.  The backward's memory is the strips'
// bottom rows and checkpoints, O(Ni Nj / ck) per pair instead of a value per
// cell.

template <typename T>
struct AdjArgs {
    const PairPlan *plan;
    const int64_t *totals;
    int64_t n_pairs;
    const T *cbuf;
    const T *ckpt;   // the forward's checkpoints: [strip][step / ck][lane][K 0..R-1, Q 0..R-1]
    const T *bnd;    // the forward's bottom rows (K, Q) per column, every strip
    T *vbuf;         // per pair, per strip boundary: V of the lower strip's first row [nj],
                     // filled with the all-ones pattern first
    int *counter;
    int *status;
    T *gbar;         // dense dk/dG (unscaled), [nx][ny] per pair
    long long wait_cycles;
    int scheme;      // sigk_scheme of the forward (scheme_dcoef)
};

template <typename T, int R, int LAM>
__host__ __device__ constexpr int adj_warp_elems() {
    return NRING * 32 * (R >> LAM) + CW;
}

template <typename T, int R, int LAM>
__global__ void __launch_bounds__(STRIP_WARPS * 32) strip_adj_kernel(AdjArgs<T> a) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int CP = 32 * NG;
    constexpr int TH = 32 * R;
    constexpr int CK = strip_ck<T>();
    extern __shared__ __align__(16) unsigned char adj_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T *ringc = reinterpret_cast<T *>(adj_smem) + (size_t)warp * adj_warp_elems<T, R, LAM>();
    T *bb = ringc + NRING * CP;
    const int64_t total_strips = a.totals[TOT_STRIPS];

    for (;;) {
        int64_t gs = 0;
        if (lane == 0) gs = atomicAdd((unsigned long long *)a.counter, 1ULL);
        gs = __shfl_sync(FULL, gs, 0);
        if (gs >= total_strips) break;
        int64_t lo = 0, hi = a.n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (a.plan[mid].strip_base <= gs) lo = mid; else hi = mid - 1;
        }
        const PairPlan pp = a.plan[lo];
        const int s = pp.ns - 1 - (int)(gs - pp.strip_base);   // last strip first
        const int nj = pp.nj;
        const int tend = nj + TH - 1;
        const int nwin = (tend + S - 1) / S;
        const int nck = (tend + CK - 1) / CK;
        const T *blk = a.cbuf + pp.c_off + (int64_t)s * pp.nw * CP;
        const T *ck = a.ckpt + pp.s_off + (int64_t)s * nck * TH * 2 + lane * (2 * R);
        const T *topb = s > 0 ? a.bnd + pp.bnd_off + (int64_t)(s - 1) * nj * 2 : nullptr;
        const T *botb = a.bnd + pp.bnd_off + (int64_t)s * nj * 2;
        const T *below = s < pp.ns - 1 ? a.vbuf + pp.bnd_off / 2 + (int64_t)s * nj : nullptr;
        T *above = s > 0 ? a.vbuf + pp.bnd_off / 2 + (int64_t)(s - 1) * nj : nullptr;
        const int prow0 = s * CP - (pp.pad >> LAM);

        T A[R], V[R], cp[R], cn[NG], co[NG], gN[NG], gO[NG];
        T KS[R], QS[R];   // the forward state after the step about to be undone
#pragma unroll
        for (int r = 0; r < R; ++r) { A[r] = 0; V[r] = 0; cp[r] = 0; KS[r] = 1; QS[r] = 0; }
        // the bottom rows the undo reads (the upper strip's K at column t for
        // lane 0, this strip's (K, Q) at column t - 32 R for lane 31), 32
        // columns a chunk, lane j holding column 32 c + j: the chunk in use
        // and the next one down, loaded a chunk ahead and read by shuffles
        T topc = 1, topn = 1, bKc = 1, bQc = 0, bKn = 1, bQn = 0;
        int tchunk = -1, bchunk = -1;
        auto top_chunk = [&](int c) -> T {
            const int col = c * 32 + lane;
            return (topb && col >= 0 && col < nj) ? topb[(int64_t)col * 2] : (T)1;
        };
        auto bot_chunk = [&](int c, T &k, T &q) {
            const int col = c * 32 + lane;
            k = (col >= 0 && col < nj) ? botb[(int64_t)col * 2] : (T)1;
            q = (col >= 0 && col < nj) ? botb[(int64_t)col * 2 + 1] : (T)0;
        };
#pragma unroll
        for (int g = 0; g < NG; ++g) { gN[g] = 0; gO[g] = 0; }
        bool timed_out = false;

        // the row below's V in chunks counted from the right, chunk c holding
        // columns nj - 1 - c CW - lane: loaded half a chunk before it is
        // published to the warp, and again, within the wait bound, while some
        // lane still sees the unwritten pattern (as in the forward)
        T vn = 0;
        auto load_below = [&](int c) {
            const int col = nj - 1 - c * CW - lane;
            vn = col >= 0 ? ld_relaxed(below + col) : (T)0;
        };
        auto wait_below = [&](int c) {
            const long long t0 = clock64();
            while (!timed_out && __any_sync(FULL, unwritten(vn))) {
                if (__any_sync(FULL, clock64() - t0 > a.wait_cycles)) {
                    timed_out = true;
                    if (lane == 0) atomicExch(a.status, (int)SIGK_ETIMEOUT);
                    break;
                }
                __nanosleep(100);
                load_below(c);
            }
        };
        if (below) {
            // start once chunks 0 and 1 are written
            load_below(0);
            wait_below(0);
            bb[lane] = vn;
            __syncwarp();
            if (CW < nj) {
                load_below(1);
                wait_below(1);
            }
        }

        // coefficient diagonals nwin-1 .. nwin-NRING+1, then one per window
#pragma unroll
        for (int k = 0; k < NRING - 1; ++k) {
            const int dg = nwin - 1 - k;
            if (dg >= 0 && dg < pp.nw)
                ring_fetch<T, NG>(&ringc[((dg + NRING) % NRING) * CP + lane * NG], blk + (int64_t)dg * CP + lane * NG);
        }
        ring_commit();
        ring_wait<0>();
        {
            const T *cw = &ringc[((nwin - 1 + NRING) % NRING) * CP + lane * NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) co[g] = cw[g];
        }
        for (int w = nwin - 1; w >= 0; --w) {
            // diagonal w - (NRING - 1) joins the ring; diagonal w - 1 was
            // fetched NRING - 1 windows ago
            {
                const int k = w - (NRING - 1);
                if (k >= 0)
                    ring_fetch<T, NG>(&ringc[(k % NRING) * CP + lane * NG], blk + (int64_t)k * CP + lane * NG);
                ring_commit();
                ring_wait<1>();
            }
#pragma unroll
            for (int g = 0; g < NG; ++g) cn[g] = co[g];
            if (w >= 1) {
                const T *cw = &ringc[((w - 1) % NRING) * CP + lane * NG];
#pragma unroll
                for (int g = 0; g < NG; ++g) co[g] = cw[g];
            } else {
#pragma unroll
                for (int g = 0; g < NG; ++g) co[g] = 0;
            }
#pragma unroll
            for (int jj = S - 1; jj >= 0; --jj) {
                const int t = w * S + jj;
                if (t >= tend) continue;
                // the forward state after step t: a checkpoint, or the last undo
                if ((t + 1) % CK == 0 || t == tend - 1) {
                    const T *src = ck + (int64_t)(t / CK) * TH * 2;
#pragma unroll
                    for (int r = 0; r < R; ++r) { KS[r] = src[r]; QS[r] = src[R + r]; }
                }
                const int col31 = t - (TH - 1);   // zero-based column of the strip's last row
                if (below && col31 >= 0 && col31 < nj - CW) {
                    // chunk c = (nj-1-col31)/CW (c >= 1) was loaded half a chunk
                    // ago: publish it; load chunk c + 1 half a chunk on
                    const int off = nj - 1 - col31, c = off / CW;
                    if (off % CW == 0) {
                        wait_below(c);
                        __syncwarp();
                        bb[lane] = vn;
                        __syncwarp();
                    } else if (off % CW == CW / 2 && (c + 1) * CW < nj) {
                        load_below(c + 1);
                    }
                }
                T vbel;
                if (below)
                    vbel = (col31 >= 0 && col31 < nj) ? bb[(nj - 1 - col31) % CW] : (T)0;
                else
                    vbel = (col31 == nj - 1) ? (T)1 : (T)0;   // seed: V(Ni+1, Nj) = 1
                const T vnext = __shfl_down_sync(FULL, V[0], 1);
                // ---- undo step t: K(a,b-1) = K - Q and the cells' sums
                T KL[R], sm[R], cw[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int g = r / S, sr = r % S;
                    cw[r] = (jj >= sr) ? cn[g] : co[g];
                    KL[r] = KS[r] - QS[r];
                }
                if ((t >> 5) != tchunk) {   // warp-uniform: a new chunk of the upper strip's row
                    const int tc = t >> 5;
                    topc = tchunk == tc + 1 ? topn : top_chunk(tc);
                    topn = top_chunk(tc - 1);
                    tchunk = tc;
                }
                const T topv = __shfl_sync(FULL, topc, t & 31);
                T kup = __shfl_up_sync(FULL, KL[R - 1], 1);
                if (lane == 0)   // row 0 of the strip is at column t: the row above is the upper strip's
                    kup = topb ? topv : (T)1;
                sm[0] = KL[0] + kup;
#pragma unroll
                for (int r = 1; r < R; ++r) sm[r] = KL[r] + KL[r - 1];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T cown = cw[r];
                    const T vb = r < R - 1 ? V[r < R - 1 ? r + 1 : 0] : (lane == 31 ? vbel : vnext);
                    const T P = vb + cp[r] * A[r];
                    const T An = A[r] + P;
                    V[r] = P + cown * An;
                    A[r] = An;
                    cp[r] = cown;
                    const int g = r / S, sr = r % S;
                    if (jj >= sr) gN[g] += An * sm[r]; else gO[g] += An * sm[r];
                }
                // ---- the state before step t: Q from the row below's update
                const T qx = QS[0] - cw[0] * sm[0];   // the row above's Q, for lane - 1
                const T qlast = __shfl_down_sync(FULL, qx, 1);
                const int bc = col31 - 1;   // the last row's column before step t
                T bkv = 1, bqv = 0;
                if (bc >= 0) {   // warp-uniform
                    if ((bc >> 5) != bchunk) {
                        const int bq = bc >> 5;
                        if (bchunk == bq + 1) { bKc = bKn; bQc = bQn; } else bot_chunk(bq, bKc, bQc);
                        bot_chunk(bq - 1, bKn, bQn);
                        bchunk = bq;
                    }
                    bkv = __shfl_sync(FULL, bKc, bc & 31);
                    bqv = __shfl_sync(FULL, bQc, bc & 31);
                }
#pragma unroll
                for (int r = 0; r < R - 1; ++r) QS[r] = QS[r + 1] - cw[r + 1] * sm[r + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) KS[r] = KL[r];
                if (lane == 31) {
                    // the strip's last row: its own bottom row, kept by the
                    // forward (beyond the grid's last column every value is
                    // virtual and meets only zero adjoints)
                    if (bc < 0) {
                        KS[R - 1] = 1;
                        QS[R - 1] = 0;
                    } else if (bc < nj) {
                        KS[R - 1] = bkv;
                        QS[R - 1] = bqv;
                    } else {
                        QS[R - 1] = 0;
                    }
                } else {
                    QS[R - 1] = qlast;
                }
                // lane 0's first row is at column t: its V goes to the strip above
                if (above && lane == 0 && t < nj) st_boundary(above + t, V[0]);
            }
            // diagonal w is complete for every group of the lane
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int p = prow0 + NG * lane + g, q = w - NG * lane - g;
                if (p >= 0 && p < pp.nx && q >= 0 && q < pp.ny)
                    a.gbar[pp.g_off + (int64_t)p * pp.ny + q] =
                        a.scheme != SIGK_SCHEME_EXPLICIT ? gN[g] * scheme_dcoef(cn[g], a.scheme) : gN[g];
                gN[g] = gO[g];
                gO[g] = 0;
            }
        }
        ring_wait<0>();
    }
}

// Chain rule through G(p,q) = <dx_p, dy_q>: dk/d dx_p = f sum_q Gbar(p,q) dy_q,
// dk/d dy_q = f sum_p Gbar(p,q) dx_p (f = incoming gradient x 1/2 4^-lambda),
// then to the points, atomically (a path appears in many pairs).  Both
// contractions run on 64 x 64 tiles of Gbar staged in shared memory; thread
// (t / 8, t % 8) owns rows t/8 and t/8 + 32 of the output tile and 4
// channels of a 32-channel block.  A block takes one (pair, contraction,
// 64-row output tile, channel block) and walks the reduction: blockIdx.y
// strides over the pairs, blockIdx.x over a pair's tiles, so a few long
// pairs still fill the GPU.
constexpr int CT = 64;

template <typename T>
__global__ void __launch_bounds__(256) grad_chain_kernel(PairSrc src, const PairPlan *plan,
                                                         int64_t n_pairs, const T *gbar,
                                                         const T *incA, const T *incB, const T *gout,
                                                         T *dA, T *dB, T scale) {
    using V4 = typename Vec4<T>::type;
    // rows padded by one element against bank conflicts, except in double
    // precision, where the padding would pass the 48 KB static limit
    constexpr int GP = sizeof(T) == 4 ? CT + 1 : CT;
    __shared__ T Gs[CT][GP];
    __shared__ V4 Vs[CT][8];
    const int64_t d = src.d;
    const int64_t D4 = (d + 3) / 4;
    const int rt = threadIdx.x >> 3, ct = threadIdx.x & 7;
    const int ncb = (int)((D4 + 7) / 8);
    for (int64_t k = blockIdx.y; k < n_pairs; k += gridDim.y) {
        const PairPlan pp = plan[k];
        if (pp.ns == 0) continue;
        const T f = gout[pp.out0] * scale;
        const T *G = gbar + pp.g_off;
        const V4 *xi = reinterpret_cast<const V4 *>(pp.swap ? incB : incA) + pp.a_row0 * D4;
        const V4 *yi = reinterpret_cast<const V4 *>(pp.swap ? incA : incB) + pp.b_row0 * D4;
        T *gx = pp.swap ? dB : dA;
        T *gy = pp.swap ? dA : dB;
        const int tx = (pp.nx + CT - 1) / CT, ty = (pp.ny + CT - 1) / CT;
        for (int64_t wi = blockIdx.x; wi < (int64_t)(tx + ty) * ncb; wi += gridDim.x) {
            // pass 0: rows p of dk/d dx, contracting over q; pass 1: rows q of dk/d dy over p
            const int pass = wi < (int64_t)tx * ncb ? 0 : 1;
            const int rem = (int)(pass == 0 ? wi : wi - (int64_t)tx * ncb);
            T *gout_pts = pass == 0 ? gx : gy;
            if (!gout_pts) continue;
            gout_pts += (pass == 0 ? pp.a_row0 : pp.b_row0) * d;
            const int nrow = pass == 0 ? pp.nx : pp.ny, nred = pass == 0 ? pp.ny : pp.nx;
            const V4 *other = pass == 0 ? yi : xi;
            {
                const int r0 = (rem / ncb) * CT;
                const int64_t cb = (int64_t)(rem % ncb) * 8;
                {
                    T acc[2][4];
                    for (int i = 0; i < 2; ++i)
                        for (int e = 0; e < 4; ++e) acc[i][e] = 0;
                    for (int k0 = 0; k0 < nred; k0 += CT) {
                        __syncthreads();
                        // Gs[i][j] = Gbar(output row r0+i, reduction index k0+j)
                        for (int u = threadIdx.x; u < CT * CT; u += blockDim.x) {
                            const int i = u / CT, j = u % CT;
                            const int orow = r0 + i, red = k0 + j;
                            T v = 0;
                            if (orow < nrow && red < nred)
                                v = pass == 0 ? G[(int64_t)orow * pp.ny + red] : G[(int64_t)red * pp.ny + orow];
                            Gs[i][j] = v;
                        }
                        for (int u = threadIdx.x; u < CT * 8; u += blockDim.x) {
                            const int j = u / 8, c4 = u % 8;
                            V4 v;
                            v.x = 0; v.y = 0; v.z = 0; v.w = 0;
                            if (k0 + j < nred && cb + c4 < D4) v = other[(int64_t)(k0 + j) * D4 + cb + c4];
                            Vs[j][c4] = v;
                        }
                        __syncthreads();
#pragma unroll 8
                        for (int j = 0; j < CT; ++j) {
                            const T g0 = Gs[rt][j], g1 = Gs[rt + 32][j];
                            const V4 v = Vs[j][ct];
                            acc[0][0] = fma(g0, v.x, acc[0][0]);
                            acc[0][1] = fma(g0, v.y, acc[0][1]);
                            acc[0][2] = fma(g0, v.z, acc[0][2]);
                            acc[0][3] = fma(g0, v.w, acc[0][3]);
                            acc[1][0] = fma(g1, v.x, acc[1][0]);
                            acc[1][1] = fma(g1, v.y, acc[1][1]);
                            acc[1][2] = fma(g1, v.z, acc[1][2]);
                            acc[1][3] = fma(g1, v.w, acc[1][3]);
                        }
                    }
                    for (int i = 0; i < 2; ++i) {
                        const int orow = r0 + rt + 32 * i;
                        if (orow >= nrow) continue;
                        for (int e = 0; e < 4; ++e) {
                            const int64_t c = (cb + ct) * 4 + e;
                            if (c >= d) continue;
                            const T v = acc[i][e] * f;
                            atomicAdd(&gout_pts[(int64_t)(orow + 1) * d + c], v);
                            atomicAdd(&gout_pts[(int64_t)orow * d + c], -v);
                        }
                    }
                }
            }
        }
    }
}

// ---- coefficients on the tensor cores (f32 paths, d >= 32) -----------------
// The same blocks as coef_kernel, from warp-level TF32 MMAs (m16n8k8) with each
// operand split x = hi + lo (hi = x rounded to TF32, lo = the remainder rounded
// to TF32) and the product taken as hi*hi + hi*lo + lo*hi: the dropped lo*lo
// term is below FP32 rounding, so the coefficients keep FP32 accuracy (a
// single TF32 product would not: about 3e-4 relative per coefficient).  A
// 64 x 64 anti-diagonal tile (diagonals W, rows P) needs c(p, q) on the
// 64 x 128 rectangle p in [P0, P0+64), q in [W0-P0-63, W0-P0+65); eight warps
// compute it as 32 x 32 pieces into shared memory, and the tile is read back
// along its diagonals and stored contiguously.

constexpr int TC_CS = 130;   // row stride of the rectangle (conflict-free diagonal reads)

__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__host__ __device__ inline int tc_stride(int64_t d) { return (int)(((d + 7) / 8) * 8 + 4); }

template <int R, int LAM>
__global__ void __launch_bounds__(256) coef_tc_kernel(PairSrc src, const PairPlan *plan,
                                                      int64_t n_pairs, const int64_t *totals,
                                                      const float *incA, const float *incB,
                                                      float *cbuf) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int CP = 32 * NG;
    extern __shared__ __align__(16) float tcs[];
    const int64_t d = src.d;
    const int D4 = (int)((d + 3) / 4);
    const int d8 = (int)((d + 7) / 8) * 8;
    const int XS = tc_stride(d);                 // = d8 + 4: 4 x odd, conflict-free fragment loads
    unsigned *xh = reinterpret_cast<unsigned *>(tcs);   // 64 rows of dx, TF32 hi / lo
    unsigned *xl = xh + 64 * XS;
    unsigned *yh = xl + 64 * XS;                        // 64 new rows of dy, hi / lo
    unsigned *yl = yh + 64 * XS;
    float *cs = reinterpret_cast<float *>(yl + 64 * XS);   // rectangle ring: 64 x 128 columns
    const float scale = 0.5f / (float)(1 << (2 * LAM));
    const int64_t total_strips = totals[TOT_STRIPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int pw = 32 * (warp >> 2), qw = 16 * (warp & 3);
    for (int64_t gs = blockIdx.x; gs < total_strips; gs += gridDim.x) {
        int64_t lo = 0, hi = n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (plan[mid].strip_base <= gs) lo = mid; else hi = mid - 1;
        }
        const PairPlan pp = plan[lo];
        const int s = (int)(gs - pp.strip_base);
        const float4 *x = reinterpret_cast<const float4 *>(pp.swap ? incB : incA) + pp.a_row0 * D4;
        const float4 *y = reinterpret_cast<const float4 *>(pp.swap ? incA : incB) + pp.b_row0 * D4;
        float *blk = cbuf + pp.c_off + (int64_t)s * pp.nw * CP;
        const int prow0 = s * CP - (pp.pad >> LAM);
        for (int P0 = 0; P0 < CP; P0 += 64) {
            const bool rows_empty = prow0 + P0 + 63 < 0 || prow0 + P0 >= pp.nx;
            __syncthreads();
            // dx rows of this row block, split once
            for (int u = threadIdx.x; u < 64 * (d8 / 4); u += blockDim.x) {
                const int i = u / (d8 / 4), c4 = u - i * (d8 / 4);
                const int p = prow0 + P0 + i;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p >= 0 && p < pp.nx && c4 < D4) v = x[(int64_t)p * D4 + c4];
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned h = to_tf32(e[k]);
                    xh[i * XS + 4 * c4 + k] = h;
                    xl[i * XS + 4 * c4 + k] = to_tf32(e[k] - __uint_as_float(h));
                }
            }
            // rectangle column block j covers q in [P0-63+64(j-1)... ]: block of columns
            // qb = W0 - P0 - 63 + 64 h, h = 0, 1; the ring keeps the two halves
            int have = -1;   // half index (in units of 64 columns from q = -P0-63) computed last
            for (int W0 = 0; W0 < pp.nw; W0 += 64) {
                const int qlo = W0 - (P0 + 63), qhi = W0 + 63 - P0;
                if (rows_empty || qhi < 0 || qlo >= pp.ny) {
                    for (int u = threadIdx.x; u < 64 * 64; u += blockDim.x) {
                        const int W = W0 + u / 64, P = P0 + (u % 64);
                        if (W < pp.nw && P < CP) blk[(int64_t)W * CP + P] = 0.f;
                    }
                    continue;
                }
                // this tile needs halves hw = W0/64 and hw + 1 (columns q = -P0-63 + 64 h + c)
                const int hw = W0 / 64;
                for (int h = hw; h <= hw + 1; ++h) {
                    if (h <= have) continue;
                    __syncthreads();
                    const int qb = -P0 - 63 + 64 * h;
                    for (int u = threadIdx.x; u < 64 * (d8 / 4); u += blockDim.x) {
                        const int i = u / (d8 / 4), c4 = u - i * (d8 / 4);
                        const int q = qb + i;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (q >= 0 && q < pp.ny && c4 < D4) v = y[(int64_t)q * D4 + c4];
                        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const unsigned hh = to_tf32(e[k]);
                            yh[i * XS + 4 * c4 + k] = hh;
                            yl[i * XS + 4 * c4 + k] = to_tf32(e[k] - __uint_as_float(hh));
                        }
                    }
                    __syncthreads();
                    float acc[2][2][4];
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
                    for (int k0 = 0; k0 < d8; k0 += 8) {
                        unsigned ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
                        for (int mi = 0; mi < 2; ++mi) {
                            const int r0 = (pw + 16 * mi + g) * XS + k0 + t, r1 = r0 + 8 * XS;
                            ah[mi][0] = xh[r0]; ah[mi][1] = xh[r1]; ah[mi][2] = xh[r0 + 4]; ah[mi][3] = xh[r1 + 4];
                            al[mi][0] = xl[r0]; al[mi][1] = xl[r1]; al[mi][2] = xl[r0 + 4]; al[mi][3] = xl[r1 + 4];
                        }
#pragma unroll
                        for (int ni = 0; ni < 2; ++ni) {
                            const int r = (qw + 8 * ni + g) * XS + k0 + t;
                            bh[ni][0] = yh[r]; bh[ni][1] = yh[r + 4];
                            bl[ni][0] = yl[r]; bl[ni][1] = yl[r + 4];
                        }
#pragma unroll
                        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                            for (int ni = 0; ni < 2; ++ni) {
                                mma_tf32(acc[mi][ni], al[mi], bh[ni]);
                                mma_tf32(acc[mi][ni], ah[mi], bl[ni]);
                                mma_tf32(acc[mi][ni], ah[mi], bh[ni]);
                            }
                    }
                    const int cbase = 64 * (h & 1);
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 2; ++ni) {
                            const int r = pw + 16 * mi + g, c = cbase + qw + 8 * ni + 2 * t;
                            cs[r * TC_CS + c] = acc[mi][ni][0];
                            cs[r * TC_CS + c + 1] = acc[mi][ni][1];
                            cs[(r + 8) * TC_CS + c] = acc[mi][ni][2];
                            cs[(r + 8) * TC_CS + c + 1] = acc[mi][ni][3];
                        }
                    have = h;
                }
                __syncthreads();
                // the diagonal tile: (W, P) -> q = W - P = -P0-63 + 64 hw + (Wl - Pl + 63)
                for (int u = threadIdx.x; u < 64 * 64; u += blockDim.x) {
                    const int Pl = u % 64, Wl = u / 64;
                    const int W = W0 + Wl, P = P0 + Pl;
                    const int col = (64 * hw + Wl - Pl + 63) & 127;   // ring column
                    if (W < pp.nw && P < CP)
                        blk[(int64_t)W * CP + P] = scheme_coef(cs[Pl * TC_CS + col] * scale, src.scheme);
                }
            }
        }
    }
}

// ---- coefficients on the fifth-generation tensor cores (tcgen05, f32, d <= 64) ----
// The same blocks as coef_kernel: d(W, P) = c(prow0 + P, W - P) for W < nw,
// P < CP.  A block of 256 threads takes a 128-row slice of a strip's coarse
// rows (the row increments, pre-scaled by 1/2 4^-lambda, split into TF32 hi
// and lo parts once) and walks the columns in chunks of 128, chunk c covering
// q = qfirst + 128 c .. + 127 with qfirst = -(P0 + 127): the chunk's column
// increments are split and staged and one thread issues the split-TF32 MMAs
// into one of three 128-column TMEM accumulators.  Diagonal block m
// (W = 128 m .. 128 m + 127 of all 128 slice rows) is then exactly the part of
// chunk m on or right of each row's diagonal (row Pl: its last Pl + 1
// columns) and the rest of chunk m + 1 (its first 127 - Pl columns).  Once
// chunk m + 1's MMAs are done, chunk m + 2's are issued, the warps read the two
// parts back into a diagonal-major shared tile St[W - 128 m][Pl] (each thread
// its own row: scalar stores, conflict-free with a row stride of 128 floats)
// and every diagonal leaves as one contiguous run of 128 floats, float4 a
// lane, through the scheme's map.  Cells outside the grid are zero (zero increments; chunks outside the
// grid skip their MMAs and read back as zero).  Waits on the MMA barrier are
// bounded: on expiry the block records SIGK_ETIMEOUT and stops.
constexpr int TC5_M = 128, TC5_N = 128, TC5_SS = 128;
constexpr int TC5_T = 256;                                     // threads: two per operand row
constexpr int TC5_NACC = 3;                                    // accumulators in flight

__host__ __device__ inline int tc5_k(int64_t d) { return (int)(((d + 3) / 4 * 4 + 7) / 8 * 8); }
inline int tc5_smem_bytes(int64_t d) { return 4 * TC5_M * tc5_k(d) * 4 + TC5_N * TC5_SS * 4; }

// Half of a row (K/8 float4s from k4 = h * K/8) of increments into registers.
__device__ __forceinline__ void tc5_fetch(float4 (&v)[8], const float4 *src, int h, int K, int k4n) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k4 = h * (K / 8) + i;
        v[i] = (src && i < K / 8 && k4 < k4n) ? __ldg(src + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
template <int R, int LAM>
__global__ void __launch_bounds__(TC5_T, 1) coef_tc5_kernel(PairSrc src, const PairPlan *plan, int64_t n_pairs,
                                                           const int64_t *totals, const float *incA,
                                                           const float *incB, float *cbuf, int *status,
                                                           long long max_wait) {
    constexpr int S = 1 << LAM;
    constexpr int CP = 32 * (R / S);
    constexpr int RB = CP >= TC5_M ? CP / TC5_M : 1;   // 128-row slices per strip
    static_assert(CP % 4 == 0, "float4 rows of a diagonal");
    extern __shared__ __align__(1024) unsigned char tc5_sm[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_slot;
    const int K = tc5_k(src.d);
    const int D4 = (int)((src.d + 3) / 4);
    unsigned char *ah = tc5_sm, *al = ah + TC5_M * K * 4;
    unsigned char *bh = al + TC5_M * K * 4, *bl = bh + TC5_N * K * 4;
    float *St = reinterpret_cast<float *>(bl + TC5_N * K * 4);   // [diagonal][slice row]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (TC5_M - 1), half = tid >> 7;   // operand row and half of K this thread stages
    const int qw = warp & 3, hsel = warp >> 2;            // TMEM lane quarter, which of its two warps
    const int Pl = qw * 32 + lane;                        // the slice row this thread reads back
    const float scale = 0.5f / (float)(1 << (2 * LAM));
    const unsigned idesc = tc5::idesc_tf32(TC5_M, TC5_N);

    if (warp == 0) tc5::alloc(&tmem_slot, 512);   // three 128-column accumulators (a power of two)
    if (tid == 0) tc5::mbar_init(&mbar);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const unsigned tmem = tmem_slot;
    unsigned phase = 0;
    bool failed = false;

    const int64_t items = totals[TOT_STRIPS] * RB;
    for (int64_t it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const int64_t gs = it / RB;
        const int rb = (int)(it - gs * RB);
        int64_t lo = 0, hi = n_pairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (plan[mid].strip_base <= gs) lo = mid; else hi = mid - 1;
        }
        const PairPlan pp = plan[lo];
        const int s = (int)(gs - pp.strip_base);
        const float4 *x = reinterpret_cast<const float4 *>(pp.swap ? incB : incA) + pp.a_row0 * D4;
        const float4 *y = reinterpret_cast<const float4 *>(pp.swap ? incA : incB) + pp.b_row0 * D4;
        float *blk = cbuf + pp.c_off + (int64_t)s * pp.nw * CP;
        const int P0 = rb * TC5_M;
        const int prow0 = s * CP - (pp.pad >> LAM) + P0;   // coarse row of slice row 0
        const bool rows_empty = prow0 + TC5_M - 1 < 0 || prow0 >= pp.nx;
        const int qfirst = -(P0 + TC5_M - 1);
        const int nblk = (pp.nw + TC5_N - 1) / TC5_N;      // diagonal blocks
        const int nch = nblk + 1;                           // chunks
        // chunk c has an accumulator (its columns meet the grid)
        auto live = [&](int c) {
            const int q0 = qfirst + c * TC5_N;
            return c < nch && !rows_empty && q0 + TC5_N - 1 >= 0 && q0 < pp.ny;
        };
        float4 nb[8];   // the next chunk's column increments, fetched ahead
        __syncthreads();
        {
            const int p = prow0 + row;
            float4 av[8];
            tc5_fetch(av, (!rows_empty && p >= 0 && p < pp.nx && P0 + row < CP) ? x + (int64_t)p * D4 : nullptr,
                      half, K, D4);
            tc5::store_half(ah, al, row, half, K, av, scale);
            const int q = qfirst + row;
            tc5_fetch(nb, (live(0) && q >= 0 && q < pp.ny) ? y + (int64_t)q * D4 : nullptr, half, K, D4);
        }
        auto issue = [&](int c) {   // stage chunk c's column increments (in nb), start its MMAs
            tc5::store_half(bh, bl, row, half, K, nb, 1.f);
            tc5::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc5::fence_after();
                tc5::gemm_split(tmem + (unsigned)((c % TC5_NACC) * TC5_N), ah, al, bh, bl, K, idesc, false);
                tc5::commit(&mbar);
            }
        };
        auto fetch_chunk = [&](int c) {
            const int qn = qfirst + c * TC5_N, q = qn + row;
            tc5_fetch(nb, (live(c) && q >= 0 && q < pp.ny) ? y + (int64_t)q * D4 : nullptr, half, K, D4);
        };
        // chunk c's MMAs done (block-uniform result; false after a timeout)
        auto wait_chunk = [&](int c) {
            if (!live(c)) return true;
            const bool ok = tc5::mbar_wait(&mbar, phase, max_wait);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(status, (int)SIGK_ETIMEOUT);
                return false;
            }
            phase ^= 1;
            tc5::fence_after();
            return true;
        };
        if (live(0)) issue(0);
        fetch_chunk(1);
        if (!wait_chunk(0)) { failed = true; break; }
        if (live(1)) issue(1);
        fetch_chunk(2);
        for (int m = 0; m < nblk; ++m) {
            if (!wait_chunk(m + 1)) { failed = true; break; }
            // chunk m + 2 into the accumulator chunk m - 1 used (read back last block)
            if (m + 2 < nch) {
                if (live(m + 2)) issue(m + 2);
                fetch_chunk(m + 3);
            }
            // read-back.  Row Pl = 32 qw + lane takes, from its quarter's 32-column
            // TMEM blocks, chunk m's columns 127 - Pl .. 127 and chunk m + 1's
            // 0 .. 126 - Pl.  Pieces 1 .. 3 (chunk m's blocks 4 - qw .. 3, then
            // chunk m + 1's blocks 0 .. 2 - qw) lie wholly on diagonals
            // 32 (pc - 1) + lane + 1 + k of the block; block 3 - qw of both
            // chunks splits at k = 31 - lane and both halves land on diagonal
            // (97 + lane + k) mod 128 (piece 0).  Warp hsel = 0 takes pieces 0
            // and 2, hsel = 1 pieces 1 and 3: 64 stores a thread, none masked.
            auto piece = [&](int c, int cb, float (&v)[32]) {
                if (live(c)) {
                    tc5::ld32(tmem + ((unsigned)(qw * 32) << 16) + (unsigned)((c % TC5_NACC) * TC5_N + cb * 32), v);
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] = 0.f;
                }
            };
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int pc = 2 * e + hsel;
                float v[32];
                if (pc == 0) {
                    float w[32];
                    piece(m, 3 - qw, v);
                    piece(m + 1, 3 - qw, w);
                    float *lo = St + (lane - 31) * TC5_SS + Pl;   // k >= 31 - lane: diagonal k + lane - 31
                    float *hi = St + (lane + 97) * TC5_SS + Pl;   // k < 31 - lane: diagonal k + lane + 97
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        if (k >= 31 - lane) lo[k * TC5_SS] = v[k];
                        else hi[k * TC5_SS] = w[k];
                    }
                } else {
                    const bool first = pc <= qw;                  // a block of chunk m
                    piece(first ? m : m + 1, first ? 3 - qw + pc : pc - qw - 1, v);
                    float *dst = St + (32 * (pc - 1) + lane + 1) * TC5_SS + Pl;
#pragma unroll
                    for (int k = 0; k < 32; ++k) dst[k * TC5_SS] = v[k];
                }
            }
            tc5::fence_before();
            __syncthreads();
            // write-out: warp w stores diagonals j = w, w + 8, .., 128 floats each
            if (P0 + 4 * lane < CP) {
#pragma unroll 4
                for (int j = warp; j < TC5_N; j += TC5_T / 32) {
                    const int W = m * TC5_N + j;
                    if (W < pp.nw) {
                        float4 v = *reinterpret_cast<const float4 *>(St + j * TC5_SS + 4 * lane);
                        if (src.scheme != SIGK_SCHEME_EXPLICIT) {
                            v.x = scheme_coef(v.x, src.scheme);
                            v.y = scheme_coef(v.y, src.scheme);
                            v.z = scheme_coef(v.z, src.scheme);
                            v.w = scheme_coef(v.w, src.scheme);
                        }
                        *reinterpret_cast<float4 *>(blk + (int64_t)W * CP + P0 + 4 * lane) = v;
                    }
                }
            }
            __syncthreads();
        }
    }
    // after a timeout, give the outstanding MMAs another bounded wait before
    // the accumulators are released
    if (failed) tc5::mbar_wait(&mbar, phase, max_wait);
    tc5::fence_before();
    __syncthreads();
    if (warp == 0) tc5::dealloc(tmem, 512);
}

template <typename T>
__global__ void strip_trivial_kernel(PairSrc src, int64_t n, T *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const PairRef pr = pair_ref(src, k);
        if (pr.la < 2 || pr.lb < 2) {
            out[pr.out0] = (T)1;
            if (pr.out1 >= 0) out[pr.out1] = (T)1;
        }
    }
}

}  // namespace

// ---- host side --------------------------------------------------------------

// Workspace layout (bytes, each part 256-aligned):
//   status (int) | counters (u64) | totals (5 x i64) | plan [n]
//   | coefficients [ncoef] | bottom rows [nbnd]
struct StripLayout {
    int64_t plan, coef, bnd, incA, incB, total;
    int64_t strips;   // at most this many strips (n x the longest pair's)
    // backward only
    int64_t vbuf, ckpt, gbar;
};


static int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

// Upper bounds from the longest path length (exact for uniform lengths).
// bwd: every strip keeps its bottom row (the forward only hands on ns - 1)
static StripLayout strip_layout(int64_t n, int64_t max_la, int64_t max_lb, int R, int lam,
                                int64_t es, int64_t rowsA, int64_t rowsB, int64_t D4, int shorter_rows = 0,
                                int bwd = 0) {
    const int64_t S = 1LL << lam, TH = 32LL * R, CP = 32LL * (R / S);
    int64_t lx = max_la > max_lb ? max_la : max_lb, ly = max_la > max_lb ? max_lb : max_la;
    if (shorter_rows) { const int64_t t = lx; lx = ly; ly = t; }
    const int64_t ni = (lx - 1) * S, nj = (ly - 1) * S;
    const int64_t ns = (ni + TH - 1) / TH;
    const int64_t nw = ((nj + TH - 2) >> lam) + 2;
    StripLayout L;
    int64_t off = 256 + 256 + 256;
    L.plan = off;
    off += al256(n * (int64_t)sizeof(PairPlan));
    L.coef = off;
    off += al256(n * ns * nw * CP * es);
    L.bnd = off;
    off += al256(n * (bwd ? ns : (ns > 1 ? ns - 1 : 0)) * nj * 2 * es + es);
    L.incA = off;
    off += al256(rowsA * D4 * 4 * es);
    L.incB = off;
    off += al256(rowsB * D4 * 4 * es);
    L.total = off;
    L.vbuf = L.ckpt = L.gbar = 0;
    L.strips = n * ns;
    return L;
}

static StripLayout strip_layout_bwd(int64_t n, int64_t max_la, int64_t max_lb, int R, int lam,
                                    int64_t es, int64_t rowsA, int64_t rowsB, int64_t D4) {
    StripLayout L = strip_layout(n, max_la, max_lb, R, lam, es, rowsA, rowsB, D4, 0, 1);
    const int64_t S = 1LL << lam, TH = 32LL * R;
    const int64_t lx = max_la > max_lb ? max_la : max_lb, ly = max_la > max_lb ? max_lb : max_la;
    const int64_t nx = lx - 1, ny = ly - 1, ni = nx * S, nj = ny * S;
    const int64_t ns = (ni + TH - 1) / TH;
    int64_t off = L.total;
    // indexed like the bottom rows (ns per pair; the last strip's is unused)
    L.vbuf = off;
    off += al256(n * ns * nj * es + es);
    // checkpoints: (K, Q) of the strip's 32 R rows after every ck-th step
    const int64_t ck = strip_ck_of(es);
    L.ckpt = off;
    off += al256(n * ns * ((nj + TH - 1 + ck - 1) / ck) * TH * 2 * es);
    L.gbar = off;
    off += al256(n * nx * ny * es);
    L.total = off;
    return L;
}

int64_t strip_bwd_workspace_bytes(int64_t n, int64_t max_la, int64_t max_lb, int lam, int dtype,
                                  int64_t rowsA, int64_t rowsB, int64_t d) {
    if (lam < 0 || lam > 3 || n <= 0) return 0;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    const int R = dtype == SIGK_F64 ? 8 : 16;
    return strip_layout_bwd(n, max_la, max_lb, R, lam, es, rowsA, rowsB, (d + 3) / 4).total;
}

// rows per lane of the strip path's forward: f64 8; f32 16 by default, 8 or
// 4 on request (a 256- or 128-row strip wastes less on short or uneven pairs)
bool strip_has_R(int R, int lam, int dtype) {
    if (dtype == SIGK_F64) return R == 8;
    return R == 16 || (R == 8 && lam <= 2) || (R == 4 && lam <= 1);
}

// dyadic orders 0..3, and channel counts whose coefficient tile fits shared
// memory (d <= 64 in f64, 128 in f32)
bool strip_supported(int lam, int64_t d, int dtype) {
    if (lam < 0 || lam > 3 || d < 1) return false;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    return (3 * GT - 1) * ((d + 3) / 4 + 1) * 4 * es <= 200 * 1024;
}

int64_t strip_workspace_bytes(int64_t n, int64_t max_la, int64_t max_lb, int lam, int dtype,
                              int64_t rowsA, int64_t rowsB, int64_t d, int R, int shorter_rows) {
    if (lam < 0 || lam > 3 || n <= 0 || !strip_has_R(R, lam, dtype)) return 0;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    return strip_layout(n, max_la, max_lb, R, lam, es, rowsA, rowsB, (d + 3) / 4, shorter_rows).total;
}

// The coefficient blocks: split-TF32 tensor-core MMAs for f32 with d >= 32,
// the FMA contraction otherwise (f64, or too few channels: at d = 16 the FMA
// kernel measured faster, 2.9 vs 3.2 ms on 4096 uneven pairs; at d = 64 the
// MMAs win, 10.1 vs 13.0 ms on 64 pairs of 4096 points).
// Strip layout of the RBF-lifted coefficients (rbf.cuh): coarse cell (p, q)
// is row P of strip s (p + pad / 2^lambda = s CP + P) on diagonal W = P + q.
template <typename T, int R, int LAM>
struct StripRbfLayout {
    PairSrc src;
    const PairPlan *plan;
    T *cbuf;
    struct Geo {
        const T *rows, *cols;
        int nx, ny, padc, nw;
        int64_t c_off;
    };
    __device__ Geo geo(int64_t k) const {
        const PairPlan &pp = plan[k];
        Geo g;
        // a_row0 / b_row0 are offsets into the row / column path's own array
        g.rows = (const T *)(pp.swap ? src.B : src.A) + pp.a_row0 * src.d;
        g.cols = (const T *)(pp.swap ? src.A : src.B) + pp.b_row0 * src.d;
        g.nx = pp.nx;
        g.ny = pp.ny;
        g.padc = pp.pad >> LAM;
        g.nw = pp.nw;
        g.c_off = pp.c_off;
        return g;
    }
    struct Row {
        int64_t base;   // element of (row P of its strip, diagonal 0)
    };
    __device__ Row row(const Geo &g, int p) const {
        constexpr int CP = 32 * (R >> LAM);
        const int Pa = p + g.padc, s = Pa / CP, P = Pa - s * CP;
        Row r;
        r.base = g.c_off + ((int64_t)s * g.nw + P) * CP + P;
        return r;
    }
    __device__ void store(const Geo &, const Row &r, int q, T c) const {
        constexpr int CP = 32 * (R >> LAM);
        cbuf[r.base + (int64_t)q * CP] = c;
    }
};

template <typename T, int R, int LAM>
static cudaError_t launch_coef(const PairSrc &src, const PairPlan *plan, int64_t n,
                               const int64_t *totals, const T *incA, const T *incB, T *cbuf,
                               int sms, cudaStream_t st, int coef_path, int *status, int64_t max_len,
                               int64_t coef_bytes) {
    cudaError_t e;
    if (src.kernel == SIGK_KERNEL_RBF) {
        // the lifted coefficient needs the points, not the increments
        StripRbfLayout<T, R, LAM> lay;
        lay.src = src;
        lay.plan = plan;
        lay.cbuf = cbuf;
        return launch_rbf_coef<T>(lay, n, max_len - 1, max_len - 1, src.d, src.sigma,
                                  0.5 / (double)(1LL << (2 * LAM)), src.scheme, cbuf, (size_t)coef_bytes,
                                  sms, st);
    }
    // tcgen05 for f32 with 32 <= d <= 64 (or on request, d <= 64); mma.sync
    // split-TF32 on request (or d > 64); FMA otherwise
    const bool tc5 = sizeof(T) == 4 && src.d <= 64 &&
                     (coef_path == 3 || (coef_path == 0 && src.d >= 32));
    if (tc5) {
        const int smem = tc5_smem_bytes(src.d);
        auto tk = coef_tc5_kernel<R, LAM>;
        if ((e = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        tk<<<sms, TC5_T, smem, st>>>(src, plan, n, totals, (const float *)incA, (const float *)incB,
                                     (float *)cbuf, status, 1LL << 26);
        return cudaGetLastError();
    }
    const bool tc = sizeof(T) == 4 && (coef_path == 2 || (coef_path == 0 && src.d >= 32));
    if (tc) {
        const int XS = tc_stride(src.d);
        const int smem = (4 * 64 * XS + 64 * TC_CS) * 4;
        auto tk = coef_tc_kernel<R, LAM>;
        if ((e = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        tk<<<sms * 2, 256, smem, st>>>(src, plan, n, totals, (const float *)incA, (const float *)incB,
                                       (float *)cbuf);
        return cudaGetLastError();
    }
    const int D4 = (int)((src.d + 3) / 4);
    const int smem = (GT + 2 * GT - 1) * (D4 | 1) * 4 * (int)sizeof(T);
    auto ck = coef_kernel<T, R, LAM>;
    if ((e = cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
    ck<<<sms * 4, 256, smem, st>>>(src, plan, n, totals, incA, incB, cbuf);
    return cudaGetLastError();
}

// Persistent sweep grid: every CTA resident at once (a strip only ever waits
// on an earlier strip, which some resident warp holds), and no more warps than
// there can be strips, so that the block scheduler spreads the working warps
// over the SMs.
static int strip_grid(const StripLayout &L, int sms, int per_sm) {
    const int64_t need = (L.strips + STRIP_WARPS - 1) / STRIP_WARPS;
    const int64_t full = (int64_t)sms * per_sm;
    return (int)(need < 1 ? 1 : need < full ? need : full);
}

template <typename T, int R, int LAM>
static cudaError_t launch_strip_t(const PairSrc &src, int64_t n, void *ws, T *out,
                                  long long wait_cycles, int fault_inject, cudaStream_t st,
                                  int64_t max_la, int64_t max_lb, int64_t rowsA, int64_t rowsB,
                                  int coef_path, int shorter_rows) {
    const int64_t D4 = (src.d + 3) / 4;
    const StripLayout L = strip_layout(n, max_la, max_lb, R, LAM, (int64_t)sizeof(T), rowsA, rowsB, D4,
                                       shorter_rows);
    unsigned char *w = (unsigned char *)ws;
    int *status = (int *)w;
    int *counter = (int *)(w + 256);
    int64_t *totals = (int64_t *)(w + 512);
    PairPlan *plan = (PairPlan *)(w + L.plan);
    T *cbuf = (T *)(w + L.coef);
    T *bnd = (T *)(w + L.bnd);
    T *incA = (T *)(w + L.incA);
    T *incB = (T *)(w + L.incB);
    cudaError_t e;
    if ((e = cudaMemsetAsync(w, 0, 768, st)) != cudaSuccess) return e;
    // every byte of the bottom rows to 0xff: the unwritten pattern
    if ((e = cudaMemsetAsync(bnd, 0xff, (size_t)(L.incA - L.bnd), st)) != cudaSuccess) return e;
    strip_trivial_kernel<T><<<64, 256, 0, st>>>(src, n, out);
    {
        const bool packed = src.mode == PM_VARLEN;
        const int64_t na = rowsA * D4 * 4, nbv = rowsB * D4 * 4;
        int ga = (int)((na + 255) / 256 < 4096 ? (na + 255) / 256 : 4096);
        int gb = (int)((nbv + 255) / 256 < 4096 ? (nbv + 255) / 256 : 4096);
        if (ga < 1) ga = 1;
        if (gb < 1) gb = 1;
        // the offsets' last entry is the exact row count of a packed array
        const int64_t nall = src.kbase + n;
        inc_kernel<T><<<ga, 256, 0, st>>>((const T *)src.A, rowsA, packed ? src.a_off + nall : nullptr,
                                          src.d, D4, incA);
        inc_kernel<T><<<gb, 256, 0, st>>>((const T *)src.B, rowsB, packed ? src.b_off + nall : nullptr,
                                          src.d, D4, incB);
    }
    plan_kernel<R, LAM><<<1, 512, 0, st>>>(src, n, plan, totals, shorter_rows, 0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = launch_coef<T, R, LAM>(src, plan, n, totals, incA, incB, cbuf, sms, st, coef_path, status,
                                    max_la > max_lb ? max_la : max_lb, L.bnd - L.coef)) != cudaSuccess)
        return e;
    StripArgs<T> a;
    a.src = src;
    a.plan = plan;
    a.totals = totals;
    a.n_pairs = n;
    a.cbuf = cbuf;
    a.bnd = bnd;
    a.counter = counter;
    a.status = status;
    a.out = out;
    a.wait_cycles = wait_cycles;
    a.fault_inject = fault_inject;
    a.sums = nullptr;
    auto sk = strip_kernel<T, R, LAM, false>;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sk, STRIP_WARPS * 32, 0)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    sk<<<strip_grid(L, sms, per_sm), STRIP_WARPS * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int R, int LAM>
static cudaError_t launch_strip_bwd_t(const PairSrc &src, int64_t n, void *ws, const T *gout, T *dA,
                                      T *dB, long long wait_cycles, cudaStream_t st, int64_t max_la,
                                      int64_t max_lb, int64_t rowsA, int64_t rowsB, int coef_path) {
    const int64_t D4 = (src.d + 3) / 4;
    const StripLayout L = strip_layout_bwd(n, max_la, max_lb, R, LAM, (int64_t)sizeof(T), rowsA, rowsB, D4);
    unsigned char *w = (unsigned char *)ws;
    int *status = (int *)w;
    int *counter = (int *)(w + 256);
    int *counter2 = (int *)(w + 264);
    int64_t *totals = (int64_t *)(w + 512);
    PairPlan *plan = (PairPlan *)(w + L.plan);
    T *incA = (T *)(w + L.incA);
    T *incB = (T *)(w + L.incB);
    cudaError_t e;
    if ((e = cudaMemsetAsync(w, 0, 768, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w + L.bnd, 0xff, (size_t)(L.incA - L.bnd), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w + L.vbuf, 0xff, (size_t)(L.ckpt - L.vbuf), st)) != cudaSuccess) return e;
    {
        const bool packed = src.mode == PM_VARLEN;
        const int64_t na = rowsA * D4 * 4, nbv = rowsB * D4 * 4;
        int ga = (int)((na + 255) / 256 < 4096 ? (na + 255) / 256 : 4096);
        int gb = (int)((nbv + 255) / 256 < 4096 ? (nbv + 255) / 256 : 4096);
        if (ga < 1) ga = 1;
        if (gb < 1) gb = 1;
        const int64_t nall = src.kbase + n;
        inc_kernel<T><<<ga, 256, 0, st>>>((const T *)src.A, rowsA, packed ? src.a_off + nall : nullptr,
                                          src.d, D4, incA);
        inc_kernel<T><<<gb, 256, 0, st>>>((const T *)src.B, rowsB, packed ? src.b_off + nall : nullptr,
                                          src.d, D4, incB);
    }
    plan_kernel<R, LAM><<<1, 512, 0, st>>>(src, n, plan, totals, 0, strip_ck<T>());
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = launch_coef<T, R, LAM>(src, plan, n, totals, incA, incB, (T *)(w + L.coef), sms, st,
                                    coef_path, status, max_la > max_lb ? max_la : max_lb,
                                    L.bnd - L.coef)) != cudaSuccess)
        return e;
    {
        StripArgs<T> a;
        a.src = src;
        a.plan = plan;
        a.totals = totals;
        a.n_pairs = n;
        a.cbuf = (const T *)(w + L.coef);
        a.bnd = (T *)(w + L.bnd);
        a.counter = counter;
        a.status = status;
        a.out = nullptr;
        a.wait_cycles = wait_cycles;
        a.fault_inject = 0;
        a.sums = (T *)(w + L.ckpt);
        auto sk = strip_kernel<T, R, LAM, true>;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sk, STRIP_WARPS * 32, 0)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        sk<<<strip_grid(L, sms, per_sm), STRIP_WARPS * 32, 0, st>>>(a);
    }
    {
        AdjArgs<T> a;
        a.plan = plan;
        a.totals = totals;
        a.n_pairs = n;
        a.cbuf = (const T *)(w + L.coef);
        a.ckpt = (const T *)(w + L.ckpt);
        a.bnd = (const T *)(w + L.bnd);
        a.vbuf = (T *)(w + L.vbuf);
        a.counter = counter2;
        a.status = status;
        a.gbar = (T *)(w + L.gbar);
        a.wait_cycles = wait_cycles;
        a.scheme = src.scheme;
        auto ak = strip_adj_kernel<T, R, LAM>;
        const int asmem = STRIP_WARPS * adj_warp_elems<T, R, LAM>() * (int)sizeof(T);
        if ((e = cudaFuncSetAttribute(ak, cudaFuncAttributeMaxDynamicSharedMemorySize, asmem)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ak, STRIP_WARPS * 32, asmem)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        ak<<<strip_grid(L, sms, per_sm), STRIP_WARPS * 32, asmem, st>>>(a);
    }
    const T scale = (T)0.5 / (T)(1LL << (2 * LAM));
    {
        // tiles of the longest pair in x, pairs in y
        const int64_t lx = max_la > max_lb ? max_la : max_lb;
        const int64_t tiles = 2 * ((lx - 1 + CT - 1) / CT) * ((D4 + 7) / 8);
        const dim3 grid((unsigned)(tiles < 1 ? 1 : tiles), (unsigned)(n < 65535 ? n : 65535));
        grad_chain_kernel<T><<<grid, 256, 0, st>>>(src, plan, n, (const T *)(w + L.gbar), incA, incB, gout, dA,
                                                   dB, scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_strip_bwd(const PairSrc &src, int64_t n, int lam, int dtype, void *ws,
                             const void *gout, void *dA, void *dB, long long wait_cycles,
                             cudaStream_t st, int64_t max_la, int64_t max_lb, int64_t rowsA,
                             int64_t rowsB, int coef_path) {
    if (n <= 0) return cudaSuccess;
#define SIGK_BWD_CASE(T, RR, L)                                                                   \
    return launch_strip_bwd_t<T, RR, L>(src, n, ws, (const T *)gout, (T *)dA, (T *)dB, wait_cycles, \
                                        st, max_la, max_lb, rowsA, rowsB, coef_path);
    if (dtype == SIGK_F64) {
        switch (lam) {
            case 0: SIGK_BWD_CASE(double, 8, 0)
            case 1: SIGK_BWD_CASE(double, 8, 1)
            case 2: SIGK_BWD_CASE(double, 8, 2)
            case 3: SIGK_BWD_CASE(double, 8, 3)
        }
    } else {
        switch (lam) {
            case 0: SIGK_BWD_CASE(float, 16, 0)
            case 1: SIGK_BWD_CASE(float, 16, 1)
            case 2: SIGK_BWD_CASE(float, 16, 2)
            case 3: SIGK_BWD_CASE(float, 16, 3)
        }
    }
#undef SIGK_BWD_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_strip(const PairSrc &src, int64_t n, int lam, int dtype, void *ws, void *out,
                         long long wait_cycles, int fault_inject, cudaStream_t st, int64_t max_la,
                         int64_t max_lb, int64_t rowsA, int64_t rowsB, int coef_path, int R,
                         int shorter_rows) {
    if (n <= 0) return cudaSuccess;
#define SIGK_FWD_CASE(T, RR, L)                                                                     \
    if (R == RR && lam == L)                                                                        \
        return launch_strip_t<T, RR, L>(src, n, ws, (T *)out, wait_cycles, fault_inject, st, max_la, \
                                        max_lb, rowsA, rowsB, coef_path, shorter_rows);
    if (dtype == SIGK_F64) {
        SIGK_FWD_CASE(double, 8, 0) SIGK_FWD_CASE(double, 8, 1) SIGK_FWD_CASE(double, 8, 2)
        SIGK_FWD_CASE(double, 8, 3)
    } else {
        SIGK_FWD_CASE(float, 16, 0) SIGK_FWD_CASE(float, 16, 1) SIGK_FWD_CASE(float, 16, 2)
        SIGK_FWD_CASE(float, 16, 3) SIGK_FWD_CASE(float, 8, 0) SIGK_FWD_CASE(float, 8, 1)
        SIGK_FWD_CASE(float, 8, 2) SIGK_FWD_CASE(float, 4, 0) SIGK_FWD_CASE(float, 4, 1)
    }
#undef SIGK_FWD_CASE
    return cudaErrorInvalidValue;
}

int read_status_word(void *ws, cudaStream_t st, int *status) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return SIGK_ECUDA;
    if (cudaMemcpy(status, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SIGK_ECUDA;
    return SIGK_OK;
}

}  // namespace sigk
