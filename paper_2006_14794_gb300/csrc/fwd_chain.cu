// Forward sweep, FP32, "row chain" form: one warp solves a chain of pairs of
// equal shape, with no grid and no increment Gram ever written to memory.
//
// The scheme (Sec. 3.1, explicit finite differences on P_lambda) is carried in
// its difference form.  With Q(a,b) = K(a,b) - K(a,b-1) the update
//   K(a,b) = K(a,b-1) + K(a-1,b) - K(a-1,b-1) + c (K(a,b-1) + K(a-1,b)),
//   c = 1/2 4^-lambda <dx_p, dy_q>        (remark after the scheme)
// becomes
//   Q(a,b) = Q(a-1,b) + c (K(a,b-1) + K(a-1,b)),   K(a,b) = K(a,b-1) + Q(a,b),
// which is the same arithmetic in exact terms but keeps the O(1) values out of
// the cancellation K(a,b-1) + K(a-1,b) - K(a-1,b-1); in FP32 it brings the
// corner's relative error from ~1e-4 to ~1e-6 at 508x508 cells.
//
// Layout of the work.  Lane l of a warp owns R consecutive refined rows
// ("slots" R*l .. R*l+R-1) of the 32*R-row band; row r of lane l works on
// column t - R*l - r at step t, so every cell it needs was produced one step
// earlier: K(a,b-1) by itself, K(a-1,b) and Q(a-1,b) by the row above
// (a register of the same lane, or lane l-1's last row through a shuffle).
// A row that reaches the last column starts the same row of the warp's next
// pair on the next step, so the pipeline fills once per chain, not per pair
// (the anti-diagonal parallelism of Sec. 3.1.1 with the diagonal held across
// the warp's registers).
//
// The band is padded at the top (32R - Ni virtual rows) and each row at the
// left (Tper - Nj virtual columns, Tper a multiple of R) with zero
// increments: there c = 0, so K = 1 and Q = 0 exactly and the boundary
// k(0,.) = k(.,0) = 1 flows into the real grid by itself.  The padding puts
// the terminal corner on lane 31, row R-1, at a fixed step of the macro-step
// in which that row turns over, so every branch below is resolved at compile
// time except "does this lane turn over to a new pair in this macro-step".
//
// Increments: the warp stages each pair's increments in shared memory once
// (column path: one buffer per pair in flight, XOR-swizzled so that the 32
// lanes, which read coarse columns NG apart, hit distinct banks; row path:
// read by each lane once, when it turns over to the pair, into registers).
// Each coarse-cell coefficient is formed once per lane as a d-term dot
// product when the group's first row enters the coarse column, and shared by
// the group's 2^lambda rows.
//
// Arithmetic: rows i and i + R/2 of a lane are carried as one float2, so each
// pair of rows costs one packed add, one packed fma and one packed add
// (FADD2/FFMA2: half the issue slots of scalar FP32 at the same FP32 lane
// throughput).  A macro-step's R / 2^lambda windows and their 2^lambda steps
// are unrolled (R steps of straight-line code), so the column increments'
// shift from group to group is register renaming; macro-steps are a loop.
#include <algorithm>

#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int CHAIN_WARPS = 2;   // warps per CTA

struct ChainArgs {
    PairSrc src;
    float *out;
    int64_t n_pairs, ppw;
    int Tper, vtop, NQ, NQV;
    int nby, nbx, nout;      // column / row increment buffers, output slots per warp
    int yunits, xunits;      // their sizes (float4)
    int warp_units;          // float4 units of shared memory per warp (incl. output slots)
    float scale;             // 1/2 * 4^-lambda
    // the solution surface on the sample grid (SURF instances): each lane's
    // values at the sample-grid nodes, a window row per window, in the band
    // layout with Tper/R + 1 slots per pair (the last: the pair's tail), as
    // band.cu's surface sweep writes them for its unpack kernel
    float *sband;
};

__device__ __forceinline__ int swz(int u) { return u ^ ((u >> 3) & 7); }

// Warp-cooperative staging of pair `kg`: the column path's NQ coarse
// increments into ybuf (NQV leading virtual ones are zero), the row path's
// 32*NG coarse increments into xbuf (leading virtual ones are zero), channels
// >= d zero; and the pair's output slots.
template <int NG, int D4>
__device__ void load_pair(float4 *ybuf, float4 *xbuf, long long *outs, const ChainArgs &a,
                          int64_t kg, int lane, int vrows) {
    const PairRef pr = pair_ref(a.src, kg);
    const int d = (int)a.src.d;
    const float *y = (const float *)a.src.B + pr.b_row0 * (int64_t)d;
    const float *x = (const float *)a.src.A + pr.a_row0 * (int64_t)d;
    const int ny = a.NQ * D4;
    const int nx = 32 * NG * D4;
    for (int u = lane; u < ny + nx; u += 32) {
        const bool isy = u < ny;
        const int uu = isy ? u : u - ny;
        const int q = uu / D4, c4 = uu - (uu / D4) * D4;
        const int real = isy ? q - a.NQV : q - vrows;
        const float *p0 = (isy ? y : x) + (int64_t)real * d;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (real >= 0) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c4 * 4 + e;
                if (c < d) v[e] = __ldg(p0 + d + c) - __ldg(p0 + c);
            }
        }
        (isy ? ybuf : xbuf)[swz(uu)] = make_float4(v[0], v[1], v[2], v[3]);
    }
    if (lane == 0) {
        outs[0] = pr.out0;
        outs[1] = pr.out1;
    }
}

// c = <dx, dy> with dx pre-scaled by 1/2 4^-lambda: FFMA2 over channel pairs.
template <int D4>
__device__ __forceinline__ float dot_inc(const float4 (&dx)[D4], const float4 (&v)[D4]) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int c4 = 0; c4 < D4; ++c4) {
        acc = __ffma2_rn(make_float2(dx[c4].x, dx[c4].y), make_float2(v[c4].x, v[c4].y), acc);
        acc = __ffma2_rn(make_float2(dx[c4].z, dx[c4].w), make_float2(v[c4].z, v[c4].w), acc);
    }
    return acc.x + acc.y;
}

// A window row of NG values (NH float2: groups g, g + NH) to 8- or 16-byte
// aligned memory.
template <int NG>
__device__ __forceinline__ void chain_store_window(float *dst, const float2 (&v)[NG / 2]) {
    if constexpr (NG == 8) {
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else if constexpr (NG == 4) {
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        reinterpret_cast<float2 *>(dst)[0] = v[0];
    }
}

// MINB: CTAs per SM the register allocation must allow (6 two-warp CTAs =
// 12 warps at <= 168 registers measured fastest for the 256x256 Gram; 1 where
// that cap would spill).
// IMPL: the implicit scheme's coefficient map (scheme_coef) on every coarse
// cell, a compile-time choice so that the explicit scheme's loop carries none
// of it.
// SURF: also keep the solution at the sample-grid nodes.  Row r of lane l is
// refined node row R l + r + 1 - vtop and at step j of position pos computes
// node column pos R + j - r + 1 - vpad (the previous pair's when that is <=
// 0); vtop and vpad are multiples of 2^lambda, so the node is on the sample
// grid exactly for the last row of each coarse group (r % 2^lambda =
// 2^lambda - 1) at step j % 2^lambda = 2^lambda - 2 of each window (0 at
// dyadic orders 0 and 1).  There group g of window w holds node (p + 1, q)
// (order 0: (p + 1, q + 1)) of coarse cell (p, q) = (P - vrows, Q - NQV),
// (P, Q) = (lane NG + g, pos NG + w - g): the band layout's cell, so the lane
// stores its NG values as one window row.
template <int R, int LAM, int D4, int MINB, bool IMPL, bool SURF = false>
__global__ void __launch_bounds__(CHAIN_WARPS * 32, MINB) chain_f32_kernel(ChainArgs a) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;        // coarse rows (groups) per lane = windows per macro-step
    constexpr int H = R / 2;         // rows i and i + H share a float2
    constexpr int NH = NG / 2;       // groups g and g + NH share a float2 of coefficients
    constexpr int JOUT = R - 2;      // step of the corner in a turn-over macro-step
    constexpr int SLOT = NG * NG;    // floats a lane's window rows take in a surface slot
    static_assert(R % S == 0 && NG % 2 == 0, "rows per lane: an even number of coarse rows");
    extern __shared__ float4 smem[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * CHAIN_WARPS + warp;
    const int64_t k0 = gw * a.ppw;
    if (k0 >= a.n_pairs) return;   // whole warp
    const int np = (int)min(a.ppw, a.n_pairs - k0);
    float4 *ybufs = smem + (size_t)warp * a.warp_units;
    float4 *xbufs = ybufs + (size_t)a.nby * a.yunits;
    long long *outs = reinterpret_cast<long long *>(xbufs + (size_t)a.nbx * a.xunits);
    const int TperR = a.Tper / R;
    const int vrows = a.vtop / S;
    const float scale = a.scale;

    float2 KP[H], QP[H];             // (K, Q) of rows (i, i + H)
    float2 CN[NH], CO[NH];           // coefficients of groups (g, g + NH): entered now / before
    float4 dxr[NG][D4];              // scaled row increments of the lane's coarse rows
    float4 yv[NG][D4];               // column increments each group is using (a shift register)
#pragma unroll
    for (int i = 0; i < H; ++i) { KP[i] = make_float2(1.f, 1.f); QP[i] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int g = 0; g < NH; ++g) { CN[g] = make_float2(0.f, 0.f); CO[g] = CN[g]; }
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int c4 = 0; c4 < D4; ++c4) {
            dxr[g][c4] = make_float4(0.f, 0.f, 0.f, 0.f);
            yv[g][c4] = dxr[g][c4];
        }
    float pK = 1.f, pQ = 0.f;

    load_pair<NG, D4>(ybufs, xbufs, outs, a, k0, lane, vrows);
    __syncwarp();

    // lane-local macro-step mm = m - lane; pair kl = floor(mm / TperR), pos = mm mod TperR
    int kl = (lane == 0) ? 0 : -((lane + TperR - 1) / TperR);
    int pos = -lane - kl * TperR;
    int by = ((kl % a.nby) + a.nby) % a.nby;   // buffers of pair kl
    int bx = ((kl % a.nbx) + a.nbx) % a.nbx;
    int lane0pos = 0, lane0pair = 0;            // warp-uniform
    const int64_t total_m = (int64_t)np * TperR + 32;

    for (int64_t m = 0; m < total_m; ++m) {
        if (lane0pos == TperR - 1) {
            // lane 0 starts pair lane0pair + 1 in the next macro-step: stage it.
            // Its buffers last served pair lane0pair + 1 - nby (nbx), which every
            // lane has left by now (lane 31 leaves a pair 31 macro-steps after
            // lane 0 and reads the column buffer only while inside it).
            const int kn = lane0pair + 1;
            if (kn < np)
                load_pair<NG, D4>(ybufs + (size_t)(kn % a.nby) * a.yunits,
                                  xbufs + (size_t)(kn % a.nbx) * a.xunits, outs + 2 * (kn % a.nout),
                                  a, k0 + kn, lane, vrows);
            __syncwarp();
        }
        const bool trans = (pos == 0);
        const float4 *ycol = ybufs + (size_t)by * a.yunits;
        const float4 *xrow = xbufs + (size_t)bx * a.xunits;
        const int qc = pos * NG;

#pragma unroll
        for (int w = 0; w < NG; ++w) {
            // ---- window start.  Group w's rows turn over in this window of a
            // turn-over macro-step: its row increments become the new pair's.
            if (trans) {
#pragma unroll
                for (int c4 = 0; c4 < D4; ++c4) {
                    const float4 v = xrow[swz((lane * NG + w) * D4 + c4)];
                    dxr[w][c4] = make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale);
                }
            }
            // group g enters column qc + w - g: group g-1's column of the last window
#pragma unroll
            for (int g = NG - 1; g > 0; --g)
#pragma unroll
                for (int c4 = 0; c4 < D4; ++c4) yv[g][c4] = yv[g - 1][c4];
#pragma unroll
            for (int c4 = 0; c4 < D4; ++c4) yv[0][c4] = ycol[swz((qc + w) * D4 + c4)];
#pragma unroll
            for (int g = 0; g < NH; ++g) CO[g] = CN[g];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                float c = dot_inc<D4>(dxr[g], yv[g]);
                if constexpr (IMPL) c = scheme_coef(c, SIGK_SCHEME_IMPLICIT);
                if (g < NH) CN[g].x = c; else CN[g - NH].y = c;
            }
            // ---- the window's S steps
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
                        if (j == JOUT && trans && lane == 31) {
                            const int kp = kl - 1;   // row R-1 just finished pair kp's last column
                            if (kp >= 0 && kp < np) {
                                const long long *o = outs + 2 * (kp % a.nout);
                                a.out[o[0]] = KP[i].y;
                                if (o[1] >= 0) a.out[o[1]] = KP[i].y;
                            }
                        }
                    }
                }
                if constexpr (SURF) {
                    constexpr int JS = S >= 2 ? S - 2 : 0;
                    if (jj == JS) {
                        // rows g S + S - 1 (packed with g + NH) are at their group's node
                        float2 sv[NH];
#pragma unroll
                        for (int g = 0; g < NH; ++g) sv[g] = KP[g * S + S - 1];
                        if (kl >= 0 && kl < np)
                            chain_store_window<NG>(a.sband + (((k0 + kl) * (TperR + 1) + pos) * 32 + lane) *
                                                                 (int64_t)SLOT + w * NG, sv);
                        if (trans && kl >= 1 && kl <= np)   // the previous pair's tail
                            chain_store_window<NG>(a.sband + (((k0 + kl - 1) * (TperR + 1) + TperR) * 32 + lane) *
                                                                 (int64_t)SLOT + w * NG, sv);
                    }
                }
                pK = (lane == 0) ? 1.f : shK;
                pQ = (lane == 0) ? 0.f : shQ;
            }
        }

        if (++pos == TperR) {
            pos = 0;
            ++kl;
            by = (by + 1 == a.nby) ? 0 : by + 1;
            bx = (bx + 1 == a.nbx) ? 0 : bx + 1;
        }
        if (++lane0pos == TperR) { lane0pos = 0; ++lane0pair; }
    }
}

template <int R, int LAM, int D4, int MINB>
cudaError_t launch_one(const ChainArgs &args, const ChainPlan &p, cudaStream_t st) {
    auto kern = args.sband ? chain_f32_kernel<R, LAM, D4, MINB, false, true>
                           : args.src.scheme == SIGK_SCHEME_IMPLICIT ? chain_f32_kernel<R, LAM, D4, MINB, true>
                                                                     : chain_f32_kernel<R, LAM, D4, MINB, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         p.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<p.grid, CHAIN_WARPS * 32, p.smem_bytes, st>>>(args);
    return cudaGetLastError();
}

template <int R, int LAM, int D4, int MINB>
int occupancy(int smem) {
    int nb = 0;
    auto kern = chain_f32_kernel<R, LAM, D4, MINB, false>;   // the implicit instance has the same resources
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, CHAIN_WARPS * 32, smem) != cudaSuccess)
        return 0;
    return nb;
}

// Instances: (R, lambda) with R / 2^lambda even, and D4 in {1, 2, 4} with
// (R / 2^lambda) * D4 <= 8 float4 registers of row increments.
#define SIGK_CHAIN_CASES(X)                                                                \
    X(4, 0, 1, 6) X(4, 0, 2, 6) X(4, 1, 1, 6) X(4, 1, 2, 6) X(4, 1, 4, 6) X(8, 0, 1, 6)       \
    X(8, 0, 2, 1) X(8, 1, 1, 6) X(8, 1, 2, 6) X(8, 2, 1, 6) X(8, 2, 2, 6) X(8, 2, 4, 6)       \
    X(16, 1, 1, 6) X(16, 2, 1, 6) X(16, 2, 2, 6) X(16, 3, 1, 6) X(16, 3, 2, 6) X(16, 3, 4, 6)

bool has_instance(int R, int lam, int D4) {
#define X(r, l, dd, mb) if (R == r && lam == l && D4 == dd) return true;
    SIGK_CHAIN_CASES(X)
#undef X
    return false;
}

int occupancy_of(int R, int lam, int D4, int smem) {
#define X(r, l, dd, mb) if (R == r && lam == l && D4 == dd) return occupancy<r, l, dd, mb>(smem);
    SIGK_CHAIN_CASES(X)
#undef X
    return 0;
}

}  // namespace

bool chain_geometry(int64_t La, int64_t Lb, int64_t d, int lam, ChainPlan &p, int rows_per_lane) {
    if (La < 2 || Lb < 2 || lam > 3 || d < 1) return false;
    const int64_t S = 1LL << lam;
    const int64_t Ni = S * (La - 1), Nj = S * (Lb - 1);
    int D4 = (int)((d + 3) / 4);
    if (D4 == 3) D4 = 4;
    if (D4 > 4) return false;
    int R = 0;
    for (int r : {4, 8, 16})
        if ((rows_per_lane == 0 || rows_per_lane == r) && 32 * r >= Ni && r >= 2 * S &&
            has_instance(r, lam, D4)) {
            R = r;
            break;
        }
    if (R == 0) return false;
    const int64_t Tper = ((Nj + R - 1) / R) * R;
    if (Tper < 2 * R || Tper > (1 << 20)) return false;
    const int64_t TperR = Tper / R;
    p.R = R; p.lam = lam; p.D4 = D4;
    p.Tper = (int)Tper;
    p.vpad = (int)(Tper - Nj);
    p.vtop = (int)(32 * R - Ni);
    p.NQ = (int)(Tper / S);
    p.NQV = (int)(p.vpad / S);
    // pair k+1 is staged one macro-step before lane 0 enters it, at (k+1)T - 1;
    // pair k's column buffer is read until lane 31 leaves it at (k+1)T + 30 and
    // its row buffer until lane 31 enters it at kT + 31
    p.nby = (int)(1 + (32 + TperR - 1) / TperR);
    p.nbx = (int)(1 + 32 / TperR);
    // pair k's output slots are read when lane 31 leaves it, at (k+1)T + 31
    p.nout = (int)(3 + 32 / TperR);
    p.yunits = ((p.NQ * D4 + 7) / 8) * 8;
    p.xunits = ((32 * (R >> lam) * D4 + 7) / 8) * 8;
    const int out_units = (p.nout * 2 * 8 + 15) / 16;
    p.warp_units = p.nby * p.yunits + p.nbx * p.xunits + out_units;
    const int64_t cta_smem = (int64_t)CHAIN_WARPS * p.warp_units * 16;
    if (cta_smem > 200 * 1024) return false;
    p.smem_bytes = (int)cta_smem;
    return true;
}

bool chain_plan(int64_t n_pairs, int64_t La, int64_t Lb, int64_t d, int lam, ChainPlan &p,
                int rows_per_lane) {
    if (n_pairs < 1 || !chain_geometry(La, Lb, d, lam, p, rows_per_lane)) return false;
    const int R = p.R, D4 = p.D4;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    const int per_sm = occupancy_of(R, lam, D4, p.smem_bytes);
    if (per_sm < 1) return false;
    const int64_t warps = (int64_t)sms * per_sm * CHAIN_WARPS;
    p.ppw = (n_pairs + warps - 1) / warps;
    const int64_t nwarps = (n_pairs + p.ppw - 1) / p.ppw;
    p.grid = (int)((nwarps + CHAIN_WARPS - 1) / CHAIN_WARPS);
    return true;
}

cudaError_t launch_chain_f32(const PairSrc &src, const ChainPlan &p, int64_t n_pairs, float *out,
                             cudaStream_t st, float *sband) {
    if (sband && src.scheme == SIGK_SCHEME_IMPLICIT) return cudaErrorInvalidValue;   // no such instance
    ChainArgs a;
    a.src = src;
    a.out = out;
    a.n_pairs = n_pairs;
    a.ppw = p.ppw;
    a.Tper = p.Tper;
    a.vtop = p.vtop;
    a.NQ = p.NQ;
    a.NQV = p.NQV;
    a.nby = p.nby;
    a.nbx = p.nbx;
    a.nout = p.nout;
    a.yunits = p.yunits;
    a.xunits = p.xunits;
    a.warp_units = p.warp_units;
    a.scale = 0.5f / (float)(1 << (2 * p.lam));
    a.sband = sband;
#define X(r, l, dd, mb) \
    if (p.R == r && p.lam == l && p.D4 == dd) return launch_one<r, l, dd, mb>(a, p, st);
    SIGK_CHAIN_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sigk
