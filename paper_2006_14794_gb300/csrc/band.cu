// Forward sweep, FP32, "band" form: the row-chain wavefront of fwd_chain.cu
// (one warp solves a chain of pairs of equal shape, lane l owning refined rows
// R*l .. R*l+R-1, the difference form Q(a,b) = Q(a-1,b) + c (K(a,b-1) +
// K(a-1,b)), K(a,b) = K(a,b-1) + Q(a,b) of the scheme of Sec. 3.1), with the
// coarse-cell coefficients c = 1/2 4^-lambda <dx_p, dy_q> (remark after the
// scheme) formed beforehand by a contraction kernel instead of inside the
// sweep.  That pays off when d is large: the sweep costs 3 operations per
// refined cell, an inline dot product d / 4^lambda more.
//
// The coefficient buffer is laid out for the sweep ("band" layout).  In
// macro-step pos of a pair (columns pos*NG .. pos*NG + NG - 1 of the padded
// coarse grid, NG = R / 2^lambda coarse rows per lane), window w, group g of
// lane l is at coarse cell (P, Q) = (l*NG + g, pos*NG + w - g).  Slot (pair,
// pos, lane) holds these NG x NG values as [w][g]: in each window a lane reads
// NG consecutive floats, and a warp reads 32 slots of one pair position, so
// every load is a full 32-byte sector.  Cells with Q < 0 (pos = 0, w < g) are
// the previous pair's last columns, which rows that have not turned over yet
// still need: they are stored in the next pair's slot 0, so the chain reads
// pair k's coefficients, tail included, from slots (k, 0 .. TperR - 1) and
// (k + 1, 0).  Virtual rows and columns (padding, as in fwd_chain.cu) hold 0.
#include <string.h>

#include "rbf.cuh"
#include "sigk_internal.cuh"
#include "tc5.cuh"

namespace sigk {

namespace {

constexpr int BAND_WARPS = 2;   // warps per CTA of the sweep
constexpr int BC_THREADS = 256; // threads per CTA of the contraction
constexpr int BC_DC = 32;       // channels staged per pass of the contraction

struct BandCoefArgs {
    PairSrc src;
    int64_t n_pairs;      // pairs of this launch (slot rows 0 .. n_pairs)
    int TperR, NQ, NQV, vrows;
    float scale;          // 1/2 4^-lambda
    float *band;
};

// Shared memory of the contraction: increments of one pair, channel-major.
//   dx: [BC_DC][32*NG + 4]      row P (padded, virtual rows zero)
//   dy: [BC_DC][ystride]        index Q + NG - 1 (zeros for Q < 0 and Q >= NQ)
template <int NG>
__host__ __device__ constexpr int bc_xstride() { return 32 * NG + 4; }
__host__ __device__ inline int bc_ystride(int NQ, int NG) { return ((NQ + 2 * NG + 3) / 4) * 4 + 4; }

// Position of row P of the staged row increments: with 8 rows per lane the
// two 16-byte halves of a lane's rows are swapped for lanes 4..7 of every 8,
// so the 8 lanes of a shared-memory phase read 8 distinct bank quads.
template <int NG>
__device__ __forceinline__ int bc_xpos(int P) {
    if constexpr (NG == 8) return P ^ (((P >> 5) & 1) << 2);
    else return P;
}

// Order of the groups inside a window of a slot: g and g + NG/2 side by side
// (the sweeps carry groups g and g + NG/2 as one float2).
template <int NG>
__host__ __device__ constexpr int band_gpos(int g) {
    return g < NG / 2 ? 2 * g : 2 * (g - NG / 2) + 1;
}

// One thread per slot (lane l, position pos) of the pair: the NG x NG cells
// (l*NG + g, pos*NG + w - g), each a d-term dot product of increments.
// Position TperR is the pair's tail (the cells with w < g there), written into
// slot 0 of the next pair.  Each block takes a contiguous run of pairs, so
// consecutive pairs of a Gram row share the row path and its staged
// increments.
template <int NG>
__global__ void __launch_bounds__(BC_THREADS, 2) band_coef_kernel(BandCoefArgs a) {
    extern __shared__ __align__(16) float bcs[];
    constexpr int NPP = 32 * NG;
    constexpr int XS = bc_xstride<NG>();
    constexpr int SLOT = NG * NG;
    const int YS = bc_ystride(a.NQ, NG);
    float *dxs = bcs;
    float *dys = bcs + BC_DC * XS;
    const int64_t d = a.src.d;
    const int nslots = 32 * (a.TperR + 1);
    const int64_t per = (a.n_pairs + gridDim.x - 1) / gridDim.x;
    const int64_t kbeg = (int64_t)blockIdx.x * per;
    const int64_t kend = kbeg + per < a.n_pairs ? kbeg + per : a.n_pairs;
    int64_t staged_x = -1;   // point row of the row path whose increments dxs holds (d <= BC_DC)
    for (int64_t k = kbeg; k < kend; ++k) {
        const PairRef pr = pair_ref(a.src, k);
        const float *x = (const float *)a.src.A + pr.a_row0 * d;
        const float *y = (const float *)a.src.B + pr.b_row0 * d;
        const int nx = (int)pr.la - 1, ny = (int)pr.lb - 1;   // real coarse rows / columns
        for (int base = 0; base < nslots; base += BC_THREADS) {
            const int u = base + (int)threadIdx.x;
            const int l = u & 31, pos = u >> 5;
            float acc[NG][NG];
#pragma unroll
            for (int w = 0; w < NG; ++w)
#pragma unroll
                for (int g = 0; g < NG; ++g) acc[w][g] = 0.f;
            for (int64_t c0 = 0; c0 < d; c0 += BC_DC) {
                if (d > BC_DC || base == 0) {
                    __syncthreads();
                    // stage channels c0 .. c0 + BC_DC - 1 (consecutive threads take
                    // consecutive channels of a row: coalesced loads)
                    if (d > BC_DC || staged_x != pr.a_row0) {
                        for (int v = threadIdx.x; v < BC_DC * NPP; v += BC_THREADS) {
                            const int P = v / BC_DC, c = v - (v / BC_DC) * BC_DC;
                            const int p = P - a.vrows;
                            float e = 0.f;
                            if (p >= 0 && p < nx && c0 + c < d)
                                e = __ldg(x + (int64_t)(p + 1) * d + c0 + c) - __ldg(x + (int64_t)p * d + c0 + c);
                            dxs[c * XS + bc_xpos<NG>(P)] = e;
                        }
                        staged_x = pr.a_row0;
                    }
                    for (int v = threadIdx.x; v < BC_DC * YS; v += BC_THREADS) {
                        const int iq = v / BC_DC, c = v - (v / BC_DC) * BC_DC;
                        const int q = iq - (NG - 1) - a.NQV;   // real column
                        float e = 0.f;
                        if (q >= 0 && q < ny && iq - (NG - 1) < a.NQ && c0 + c < d)
                            e = __ldg(y + (int64_t)(q + 1) * d + c0 + c) - __ldg(y + (int64_t)q * d + c0 + c);
                        dys[c * YS + iq] = e;
                    }
                    __syncthreads();
                }
                if (u < nslots) {
                    const int cn = (int)(d - c0 < BC_DC ? d - c0 : BC_DC);
#pragma unroll 2
                    for (int c = 0; c < cn; ++c) {
                        float xv[NG], yv[2 * NG];
                        const float *xr = dxs + c * XS + l * NG;
                        const float *yr = dys + c * YS + pos * NG;   // Q = pos*NG - (NG-1) + j
                        if constexpr (NG >= 4) {
                            const int sw = NG == 8 ? ((l >> 2) & 1) : 0;   // see bc_xpos
#pragma unroll
                            for (int h = 0; h < NG / 4; ++h) {
                                const float4 v = *reinterpret_cast<const float4 *>(xr + 4 * (h ^ sw));
                                xv[4 * h] = v.x; xv[4 * h + 1] = v.y; xv[4 * h + 2] = v.z; xv[4 * h + 3] = v.w;
                            }
#pragma unroll
                            for (int h = 0; h < NG / 2; ++h) {
                                const float4 v = *reinterpret_cast<const float4 *>(yr + 4 * h);
                                yv[4 * h] = v.x; yv[4 * h + 1] = v.y; yv[4 * h + 2] = v.z; yv[4 * h + 3] = v.w;
                            }
                        } else {
                            const float2 v = *reinterpret_cast<const float2 *>(xr);
                            xv[0] = v.x; xv[1] = v.y;
                            const float2 w0 = *reinterpret_cast<const float2 *>(yr);
                            const float2 w1 = *reinterpret_cast<const float2 *>(yr + 2);
                            yv[0] = w0.x; yv[1] = w0.y; yv[2] = w1.x; yv[3] = w1.y;
                        }
#pragma unroll
                        for (int w = 0; w < NG; ++w)
#pragma unroll
                            for (int g = 0; g < NG; ++g)
                                acc[w][g] = fmaf(xv[g], yv[w - g + NG - 1], acc[w][g]);
                    }
                }
            }
            if (u >= nslots) continue;
#pragma unroll
            for (int w = 0; w < NG; ++w)
#pragma unroll
                for (int g = 0; g < NG; ++g) acc[w][g] = scheme_coef(acc[w][g] * a.scale, a.src.scheme);
            if (pos < a.TperR && pos > 0) {
                float4 *dst = reinterpret_cast<float4 *>(a.band + (((k * a.TperR + pos) * 32) + l) * SLOT);
                if constexpr (NG >= 4) {
#pragma unroll
                    for (int w = 0; w < NG; ++w)
#pragma unroll
                        for (int h = 0; h < NG / 4; ++h)
                            dst[w * (NG / 4) + h] = make_float4(acc[w][2 * h], acc[w][2 * h + NG / 2],
                                                                acc[w][2 * h + 1], acc[w][2 * h + 1 + NG / 2]);
                } else {
                    dst[0] = make_float4(acc[0][0], acc[0][1], acc[1][0], acc[1][1]);
                }
            } else if (pos == 0) {
                // the pair's own cells (w >= g); the cells w < g belong to the
                // previous pair's block, which writes them (pair 0: zeros)
                float *dst = a.band + ((k * a.TperR) * 32 + l) * SLOT;
#pragma unroll
                for (int w = 0; w < NG; ++w)
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (w >= g) dst[w * NG + band_gpos<NG>(g)] = acc[w][g];
                        else if (k == 0) dst[w * NG + band_gpos<NG>(g)] = 0.f;
                    }
            } else {
                // pos == TperR: the tail (w < g) into slot 0 of the next pair; after
                // the last pair the slot has no owner, so its own cells are zeroed
                float *dst = a.band + (((k + 1) * a.TperR) * 32 + l) * SLOT;
#pragma unroll
                for (int w = 0; w < NG; ++w)
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (w < g) dst[w * NG + band_gpos<NG>(g)] = acc[w][g];
                        else if (k == a.n_pairs - 1) dst[w * NG + band_gpos<NG>(g)] = 0.f;
                    }
            }
        }
    }
}

struct BandArgs {
    PairSrc src;
    float *out;
    const float *band;
    int64_t n_pairs, ppw;
    int TperR;
    // what the adjoint needs to run the sweep backwards (null: forward only)
    float *ckpt;     // [warp][nck][lane][2R]: (K, Q) of every row after each BAND_CK-th macro-step
    float *exitk;    // [pair][lane][R]: K of each row on its pair's last column
    float *botq;     // [warp][steps + 1]: Q of the warp's last row before each step
    int nck;         // checkpoint slots per warp
    int64_t bq_stride;
    // the solution surface on the sample grid (SURF instances): each lane's
    // values at the sample-grid nodes, a window row per window, in the band
    // layout with TperR + 1 slots per pair (slot TperR: the tail); unpacked by
    // band_gbar_kernel in surface mode
    float *sband;
};

constexpr int BAND_CK = 8;   // macro-steps between checkpoints of the forward state

template <int NG>
__device__ __forceinline__ void load_window(float (&v)[NG], const float *p) {
    if constexpr (NG == 8) {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (NG == 4) {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const float2 a = __ldcs(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1] = a.y;
    }
}

// A window row of NG values (NH float2: groups g, g + NH) to 16-byte aligned
// band memory.
template <int NG>
__device__ __forceinline__ void store_window(float *dst, const float2 (&v)[NG / 2]) {
    if constexpr (NG == 8) {
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else if constexpr (NG == 4) {
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        reinterpret_cast<float2 *>(dst)[0] = v[0];
    }
}

// The sweep: fwd_chain.cu's chain_f32_kernel with its staging and dot
// products replaced by one coefficient vector per window, prefetched one
// macro-step ahead into the registers the window has just consumed.
//
// SURF: also keep the solution at the sample-grid nodes (the surface).  Row
// r of lane l, padded row R l + r, is refined node row a = R l + r + 1 - vtop;
// at step j of position pos it computes padded column pos R + j - r (the
// previous pair's when negative), node column b = that + 1 - vpad.  vtop and
// vpad are multiples of 2^lambda, so the node is on the sample grid exactly
// when a and b are: r % 2^lambda = 2^lambda - 1 (the last row of each coarse
// group), and then b = j - r + 1 = j + 2 (mod 2^lambda), i.e. at step
// j % 2^lambda = 2^lambda - 2 of each window (0 for dyadic orders 0 and 1).
// There, group g of window w holds node (p + 1, q) (dyadic order 0: (p + 1,
// q + 1)) of the coarse cell (p, q) = (P - vrows, Q - NQV), (P, Q) = (lane NG
// + g, pos NG + w - g): the band layout's cell, so the lane stores its NG
// values as one window row.
template <int R, int LAM, int MINB, bool SAVE, bool SURF = false>
__global__ void __launch_bounds__(BAND_WARPS * 32, MINB) chain_band_kernel(BandArgs a) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int H = R / 2;
    constexpr int NH = NG / 2;
    constexpr int JOUT = R - 2;
    constexpr int SLOT = NG * NG;
    static_assert(R % S == 0 && NG % 2 == 0 && NG <= 8, "2, 4 or 8 coarse rows per lane");

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * BAND_WARPS + warp;
    const int64_t k0 = gw * a.ppw;
    if (k0 >= a.n_pairs) return;   // whole warp
    const int np = (int)min(a.ppw, a.n_pairs - k0);
    const int TperR = a.TperR;

    float2 KP[H], QP[H];
    float2 CN[NH], CO[NH];
    float cb[NG][NG];   // this macro-step's coefficients [window][group]; refilled window by window
#pragma unroll
    for (int i = 0; i < H; ++i) { KP[i] = make_float2(1.f, 1.f); QP[i] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int g = 0; g < NH; ++g) { CN[g] = make_float2(0.f, 0.f); CO[g] = CN[g]; }
    float pK = 1.f, pQ = 0.f;

    // slot of local pair kk at position pp, or null outside the chain (its
    // first pair's rows before they start, and after the last pair except the
    // slot that holds that pair's tail)
    auto slot = [&](int kk, int pp) -> const float * {
        if (kk < 0 || kk > np || (kk == np && pp != 0)) return nullptr;
        return a.band + (((k0 + kk) * TperR + pp) * 32 + lane) * (int64_t)SLOT;
    };

    int kl = (lane == 0) ? 0 : -((lane + TperR - 1) / TperR);
    int pos = -lane - kl * TperR;
    {
        const float *p0 = slot(kl, pos);
#pragma unroll
        for (int w = 0; w < NG; ++w) {
            if (p0) load_window<NG>(cb[w], p0 + w * NG);
            else
#pragma unroll
                for (int g = 0; g < NG; ++g) cb[w][g] = 0.f;
        }
    }
    const int64_t total_m = (int64_t)np * TperR + 32;
    float *bq = SAVE ? a.botq + gw * a.bq_stride : nullptr;
    if (SAVE && lane == 31) bq[0] = 0.f;

    for (int64_t m = 0; m < total_m; ++m) {
        const bool trans = (pos == 0);
        const float *pn = (pos + 1 == TperR) ? slot(kl + 1, 0) : slot(kl, pos + 1);
        // exit states go to the pair the rows leave (kl - 1), when it is one of the chain's
        float *ex = (SAVE && trans && kl >= 1 && kl <= np)
                        ? a.exitk + ((k0 + kl - 1) * 32 + lane) * (int64_t)R : nullptr;

#pragma unroll
        for (int w = 0; w < NG; ++w) {
#pragma unroll
            for (int g = 0; g < NH; ++g) {
                CO[g] = CN[g];
                CN[g] = make_float2(cb[w][2 * g], cb[w][2 * g + 1]);   // groups g, g + NH
            }
            if (pn) load_window<NG>(cb[w], pn + w * NG);
            else
#pragma unroll
                for (int g = 0; g < NG; ++g) cb[w][g] = 0.f;
#pragma unroll
            for (int jj = 0; jj < S; ++jj) {
                const int j = w * S + jj;
                const float kH1 = KP[H - 1].x, qH1 = QP[H - 1].x;   // row H-1 before this step
                float shK = 0.f, shQ = 0.f;
#pragma unroll
                for (int i = H - 1; i >= 0; --i) {
                    const int g1 = i / S, s1 = i % S;   // row i; row i+H: group g1+NH, same s1
                    if (jj == s1 && trans) {            // row starts its next pair now: k(.,0) = 1
                        if (g1 == w) {
                            if (ex) ex[i] = KP[i].x;
                            KP[i].x = 1.f;
                        }
                        if (g1 + NH == w) {
                            if (ex) ex[i + H] = KP[i].y;
                            KP[i].y = 1.f;
                        }
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
                            if (kp >= 0 && kp < np && a.out) {
                                const PairRef pr = pair_ref(a.src, k0 + kp);
                                a.out[pr.out0] = KP[i].y;
                                if (pr.out1 >= 0) a.out[pr.out1] = KP[i].y;
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
                            store_window<NG>(a.sband + (((k0 + kl) * (TperR + 1) + pos) * 32 + lane) * (int64_t)SLOT +
                                                 w * NG, sv);
                        if (trans && kl >= 1 && kl <= np)   // the previous pair's tail
                            store_window<NG>(a.sband + (((k0 + kl - 1) * (TperR + 1) + TperR) * 32 + lane) *
                                                           (int64_t)SLOT + w * NG, sv);
                    }
                }
                if (SAVE && lane == 31) bq[m * R + j + 1] = QP[H - 1].y;
                pK = (lane == 0) ? 1.f : shK;
                pQ = (lane == 0) ? 0.f : shQ;
            }
        }
        if (SAVE && ((m + 1) % BAND_CK == 0 || m == total_m - 1)) {
            float4 *ck = reinterpret_cast<float4 *>(a.ckpt + ((gw * a.nck + m / BAND_CK) * 32 + lane) * (int64_t)(2 * R));
#pragma unroll
            for (int i = 0; i < H; i += 2) {
                ck[i / 2] = make_float4(KP[i].x, KP[i].y, KP[i + 1].x, KP[i + 1].y);
                ck[H / 2 + i / 2] = make_float4(QP[i].x, QP[i].y, QP[i + 1].x, QP[i + 1].y);
            }
        }
        if (++pos == TperR) {
            pos = 0;
            ++kl;
        }
    }
}

template <int NG>
cudaError_t launch_coef(const BandCoefArgs &a, int sms, cudaStream_t st) {
    const int smem = (int)sizeof(float) * BC_DC * (bc_xstride<NG>() + bc_ystride(a.NQ, NG));
    auto kern = band_coef_kernel<NG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BC_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > a.n_pairs) grid = a.n_pairs;
    kern<<<(int)grid, BC_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// The same band on the fifth-generation tensor cores (tcgen05), for d <= 64.
// A block takes a contiguous run of pairs; per pair, per 128-row tile of the
// padded rows: the row increments (scaled by 1/2 4^-lambda) are split into
// TF32 hi and lo parts and staged once, then the padded columns are walked in
// chunks of 128 (the next chunk's increments fetched while the MMAs run): one
// thread issues the split-TF32 MMA chain (D = 128 x 128 fp32 in TMEM), the
// warps copy D into a shared tile, and each warp then writes four slot
// positions of one lane block, lane (s, g) reading row l*NG + g of the tile
// along the slot's window (conflict-free with the tile stride 132) and the
// lanes of a slot storing one 32-byte window row together.  Entries outside
// the chunk, and the previous pair's cells of slot 0, are left to the chunk or
// pair that owns them; the pair's tail goes to slot 0 of the next pair.  Waits
// are bounded (status word SIGK_ETIMEOUT).
constexpr int BT5_M = 128, BT5_N = 128, BT5_SS = BT5_N + 4, BT5_T = 256;

inline int bt5_smem_bytes(int64_t d) { return 4 * BT5_M * tc5::tc5_k_of(d) * 4 + BT5_M * BT5_SS * 4; }

template <int NG>
__global__ void __launch_bounds__(BT5_T, 1) band_coef_tc5_kernel(BandCoefArgs a, int *status, long long max_wait) {
    constexpr int SLOT = NG * NG;
    constexpr int NPP = 32 * NG;          // padded rows
    constexpr int SPW = 32 / NG;          // slot positions per warp task (lane = s * NG + g)
    extern __shared__ __align__(1024) unsigned char bt5_sm[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_slot;
    const int64_t d = a.src.d;
    const int K = tc5::tc5_k_of(d);
    const int D4 = (int)((d + 3) / 4);
    unsigned char *ah = bt5_sm, *al = ah + BT5_M * K * 4;
    unsigned char *bh = al + BT5_M * K * 4, *bl = bh + BT5_N * K * 4;
    float *St = reinterpret_cast<float *>(bl + BT5_N * K * 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (BT5_M - 1), half = tid >> 7;
    const unsigned idesc = tc5::idesc_tf32(BT5_M, BT5_N);
    const int TperR = a.TperR, NQ = a.NQ;

    if (warp == 0) tc5::alloc(&tmem_slot, BT5_N);
    if (tid == 0) tc5::mbar_init(&mbar);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const unsigned tmem = tmem_slot;
    unsigned phase = 0;
    bool failed = false;

    const int64_t per = (a.n_pairs + gridDim.x - 1) / gridDim.x;
    const int64_t kbeg = (int64_t)blockIdx.x * per;
    const int64_t kend = kbeg + per < a.n_pairs ? kbeg + per : a.n_pairs;
    for (int64_t k = kbeg; k < kend && !failed; ++k) {
        const PairRef pr = pair_ref(a.src, k);
        const float *x = (const float *)a.src.A + pr.a_row0 * d;
        const float *y = (const float *)a.src.B + pr.b_row0 * d;
        const int nx = (int)pr.la - 1, ny = (int)pr.lb - 1;
        // slots no chunk writes: pair 0's slot 0 before its own cells, and the
        // last pair's tail slot after its tail
        if (k == 0 || k == a.n_pairs - 1) {
            for (int v = tid; v < 32 * SLOT; v += BT5_T) {
                const int l = v / SLOT, e = v - l * SLOT, w = e / NG, gp = e - w * NG;
                const int g = (gp & 1) ? gp / 2 + NG / 2 : gp / 2;   // inverse of band_gpos
                if (k == 0 && w < g) a.band[(int64_t)l * SLOT + e] = 0.f;
                if (k == a.n_pairs - 1 && w >= g) a.band[(((k + 1) * TperR) * 32 + l) * (int64_t)SLOT + e] = 0.f;
            }
        }
        for (int P0 = 0; P0 < NPP && !failed; P0 += BT5_M) {
            float4 nb[8];
            __syncthreads();
            {
                // the tile's row increments (padded rows P: real row P - vrows), once
                const int p = P0 + row - a.vrows;
                float4 av[8];
                const bool ok = P0 + row < NPP && p >= 0 && p < nx;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k4 = half * (K / 8) + i;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok && i < K / 8 && k4 < D4) {
                        const float *r0 = x + (int64_t)p * d + 4 * k4, *r1 = r0 + d;
                        const int c = 4 * k4;
                        v.x = c < d ? r1[0] - r0[0] : 0.f;
                        v.y = c + 1 < d ? r1[1] - r0[1] : 0.f;
                        v.z = c + 2 < d ? r1[2] - r0[2] : 0.f;
                        v.w = c + 3 < d ? r1[3] - r0[3] : 0.f;
                    }
                    av[i] = v;
                }
                tc5::store_half(ah, al, row, half, K, av, a.scale);
            }
            auto fetch_cols = [&](int Q0) {
                const int q = Q0 + row - a.NQV;
                const bool ok = Q0 < NQ && Q0 + row < NQ && q >= 0 && q < ny;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k4 = half * (K / 8) + i;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok && i < K / 8 && k4 < D4) {
                        const float *r0 = y + (int64_t)q * d + 4 * k4, *r1 = r0 + d;
                        const int c = 4 * k4;
                        v.x = c < d ? r1[0] - r0[0] : 0.f;
                        v.y = c + 1 < d ? r1[1] - r0[1] : 0.f;
                        v.z = c + 2 < d ? r1[2] - r0[2] : 0.f;
                        v.w = c + 3 < d ? r1[3] - r0[3] : 0.f;
                    }
                    nb[i] = v;
                }
            };
            fetch_cols(0);
            for (int Q0 = 0; Q0 < NQ; Q0 += BT5_N) {
                tc5::store_half(bh, bl, row, half, K, nb, 1.f);
                tc5::fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc5::fence_after();
                    tc5::gemm_split(tmem, ah, al, bh, bl, K, idesc, false);
                    tc5::commit(&mbar);
                }
                fetch_cols(Q0 + BT5_N);
                const bool ok = tc5::mbar_wait(&mbar, phase, max_wait);
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    if (tid == 0) atomicExch(status, (int)SIGK_ETIMEOUT);
                    break;
                }
                phase ^= 1;
                tc5::fence_after();
                {
                    const int r = (warp & 3) * 32 + lane, cb = (warp >> 2) * 64;
#pragma unroll
                    for (int c0 = 0; c0 < 64; c0 += 32) {
                        float v[32];
                        tc5::ld32(tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(cb + c0), v);
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(&St[r * BT5_SS + cb + c0 + j]) =
                                make_float4(scheme_coef(v[j], a.src.scheme), scheme_coef(v[j + 1], a.src.scheme),
                                            scheme_coef(v[j + 2], a.src.scheme), scheme_coef(v[j + 3], a.src.scheme));
                    }
                }
                tc5::fence_before();
                __syncthreads();
                // slots with entries in this chunk: pos in [ceil((Q0 - NG + 1) / NG), (Q0 + 127 + NG - 1) / NG]
                const int pos_lo = Q0 / NG, pos_hi = min((Q0 + BT5_N - 1 + NG - 1) / NG, TperR);
                const int l_lo = P0 / NG, l_hi = min(P0 + BT5_M, NPP) / NG;   // lane blocks of this tile
                const int npos4 = (pos_hi - pos_lo + SPW) / SPW;
                const int s = lane / NG, g = lane - s * NG;
                const int gp = band_gpos<NG>(g);
                for (int t = warp; t < (l_hi - l_lo) * npos4; t += BT5_T / 32) {
                    const int l = l_lo + t / npos4;
                    const int pos = pos_lo + (t - (t / npos4) * npos4) * SPW + s;
                    if (pos > pos_hi) continue;
                    const int P = l * NG + g;
                    const float *srow = St + (P - P0) * BT5_SS;
                    // destination slot: the pair's own, or (the tail) the next pair's slot 0
                    const bool tail = pos == TperR;
                    float *dst = a.band + ((tail ? (k + 1) * TperR : k * TperR + pos) * 32 + l) * (int64_t)SLOT + gp;
#pragma unroll
                    for (int w = 0; w < NG; ++w) {
                        const int Q = pos * NG + w - g;
                        const bool own = tail ? (w < g) : (Q >= 0);
                        if (own && Q >= Q0 && Q < Q0 + BT5_N) dst[w * NG] = srow[Q - Q0];
                    }
                }
                __syncthreads();
            }
        }
    }
    if (failed) tc5::mbar_wait(&mbar, phase, max_wait);
    tc5::fence_before();
    __syncthreads();
    if (warp == 0) tc5::dealloc(tmem, BT5_N);
}

template <int NG>
cudaError_t launch_coef_tc5(const BandCoefArgs &a, int sms, int *status, cudaStream_t st) {
    const int smem = bt5_smem_bytes(a.src.d);
    auto kern = band_coef_tc5_kernel<NG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = sms;
    if (grid > a.n_pairs) grid = a.n_pairs;
    kern<<<(int)grid, BT5_T, smem, st>>>(a, status, 1LL << 26);
    return cudaGetLastError();
}

// (R, lambda) with R / 2^lambda in {2, 4, 8}; MINB as fwd_chain.cu
#define SIGK_BAND_CASES(X) \
    X(4, 0, 6) X(4, 1, 6) X(8, 0, 6) X(8, 1, 6) X(8, 2, 6) X(16, 1, 6) X(16, 2, 6) X(16, 3, 6)

bool band_has_instance(int R, int lam) {
#define X(r, l, mb) if (R == r && lam == l) return true;
    SIGK_BAND_CASES(X)
#undef X
    return false;
}

template <int R, int LAM, int MINB>
int band_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chain_band_kernel<R, LAM, MINB, false>,
                                                      BAND_WARPS * 32, 0) != cudaSuccess)
        return 0;
    return nb;
}

int band_occupancy_of(int R, int lam) {
#define X(r, l, mb) if (R == r && lam == l) return band_occupancy<r, l, mb>();
    SIGK_BAND_CASES(X)
#undef X
    return 0;
}

// ---- the adjoint: the band sweep run backwards in time ----------------------
// The reverse mode of the difference form (as in the strip adjoint of
// fwd_strip.cu): with A(a,b) = dk/dQ(a,b) and V(a,b) = P(a,b) + c(a,b) A(a,b),
//   P(a,b) = c(a,b+1) A(a,b+1) + V(a+1,b),   A(a,b) = A(a,b+1) + P(a,b),
// A(., Nj+1) = 0, V(Ni+1, b) = [b = Nj] g (g the incoming gradient), and
// dk/dc(a,b) = A(a,b) (K(a,b-1) + K(a-1,b)).  Running the chain's schedule
// backwards (rows ascending within a step) has every input ready, as in the
// strip adjoint.  The sums K(a,b-1) + K(a-1,b) are not stored: the forward
// step is undone in place,
//   K(a,b-1) = K(a,b) - Q(a,b),   Q(a-1,b) = Q(a,b) - c(a,b) (K(a,b-1) + K(a-1,b)),
// from the state after the step, exact up to rounding, with the state reset
// to the forward's own every BAND_CK macro-steps (checkpoints), the K a row
// had when it left its pair (exit states: the forward resets K to 1 there),
// and the last row's Q before each step (it has no row below to recover it
// from).  dk/dc is summed per coarse cell in registers and stored densely.

struct BandAdjArgs {
    PairSrc src;            // oriented: rows refine the A paths
    const float *band;      // coefficients, band layout
    const float *ckpt, *exitk, *botq;
    int nck;
    int64_t bq_stride;
    const float *gout;      // incoming gradient, indexed like the forward's outputs
    float *gband;           // dk/dc (unscaled) in the band layout, TperR + 1 slots per pair
                            // (slot TperR: the pair's tail), unpacked by band_gbar_kernel
    int64_t n_pairs, ppw;
    int TperR, NQ, NQV, vrows, nx, ny;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int NBYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (NBYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(NBYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// dk/dc from the adjoint's band layout into the dense Gbar the chain-rule
// contractions read: [row path * nx][column path * ny] (Gram: every column
// path of the call; pairs: one nx x ny block per pair).  Pair k's cell (P, Q)
// = (l NG + g, Q) is in slot (k, pos) window w with pos NG + w = Q + g (slot
// TperR: the tail).  A block takes gb_pos(NG) positions of one pair: it
// stages those slots and the next one in shared memory (coalesced), then
// writes the real cells of columns Q in [pos0 NG, (pos0 + gb_pos) NG) row by
// row, each row a contiguous run (window rows staged NG + 1 floats apart):
// 32 columns (128 bytes) a row for NG <= 4, 32 for NG = 8 (four positions,
// the static shared memory's limit).
__host__ __device__ constexpr int gb_pos(int NG) { return NG <= 4 ? 8 : 4; }
constexpr int GB_THREADS = 256;
// position groups per pair: the columns Q < NQ = TperR NG, and for the
// surface also Q = NQ (its last node column, in the tail slot)
__host__ __device__ inline int gb_groups(int TperR, bool surf, int NG) {
    return (TperR + (surf ? 1 : 0) + gb_pos(NG) - 1) / gb_pos(NG);
}

struct BandGbarArgs {
    PairSrc src;
    const float *gband;
    float *gbar;
    int64_t g_ld;           // floats per gbar row
    int64_t a_first;        // first A path of this launch (rows of gbar count from it)
    int gram;               // 1: gbar columns hold every B path of the call
    int64_t n_pairs;
    int TperR, NQV, vrows, nx, ny;
    // surface mode (s_pair > 0): the band holds the sweep's values at the
    // sample-grid nodes, node (p + 1, q + q_off) of cell (p, q) (q_off = 1 at
    // dyadic order 0, where the stored node is the cell's lower-right corner;
    // 0 above, the lower-left one, the last column coming from the tail slot);
    // they go to gbar[(kbase + k) s_pair + (p + 1) s_a + (q + q_off) s_b]
    int64_t s_pair, s_a, s_b;
    int q_off;
};

template <int NG>
__global__ void __launch_bounds__(GB_THREADS) band_gbar_kernel(BandGbarArgs a) {
    constexpr int SLOT = NG * NG;
    constexpr int NP = 32 * NG;                 // padded rows
    constexpr int GB_POS = gb_pos(NG);
    constexpr int SPAN = GB_POS * NG;           // columns per block task
    constexpr int WS = NG + 1;                  // staged window row stride: consecutive
                                                // columns of a row hit distinct banks
    constexpr int SS = NG * WS;                 // staged slot stride
    __shared__ float sl[(GB_POS + 1) * 32 * SS];
    const int ngroups = gb_groups(a.TperR, a.s_pair > 0, NG);
    const int64_t tasks = a.n_pairs * ngroups;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int64_t k = t / ngroups;
        const int pos0 = (int)(t - k * ngroups) * GB_POS;
        const int npos = min(GB_POS + 1, a.TperR + 1 - pos0);   // slots pos0 .. pos0 + npos - 1
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(a.gband + ((k * (a.TperR + 1) + pos0) * 32) * (int64_t)SLOT);
        for (int v = threadIdx.x; v < npos * 32 * SLOT / 4; v += GB_THREADS) {
            const float4 x = src[v];
            const int slot = v / (SLOT / 4), e = (v - slot * (SLOT / 4)) * 4;
            float *d = sl + slot * SS;
            d[(e / NG) * WS + e % NG] = x.x;
            d[((e + 1) / NG) * WS + (e + 1) % NG] = x.y;
            d[((e + 2) / NG) * WS + (e + 2) % NG] = x.z;
            d[((e + 3) / NG) * WS + (e + 3) % NG] = x.w;
        }
        __syncthreads();
        const bool surf = a.s_pair > 0;
        float *base;
        int64_t sr = a.g_ld, sc = 1;
        if (surf) {
            base = a.gbar + (a.src.kbase + k) * a.s_pair + a.s_a;   // node row p + 1
            sr = a.s_a;
            sc = a.s_b;
        } else {
            const PairRef pr = pair_ref(a.src, k);
            const int64_t ia = pr.a_row0 / a.src.La - a.a_first;
            const int64_t jb = a.gram ? pr.b_row0 / a.src.Lb : 0;
            base = a.gbar + ia * a.nx * a.g_ld + jb * a.ny;
        }
        // surface: column 0 too when the pairs have virtual columns at the
        // left (NQV >= 1 at dyadic orders >= 1): there the stored node is the
        // boundary value, exactly 1 (c = 0 keeps K = 1 and Q = 0), and the
        // border fill need not write that strided column; without them the
        // slot holds the previous pair's last column instead
        const int qlo = surf && a.q_off == 0 && a.NQV == 0 ? 1 : 0;
        const int qhi = surf ? a.ny - a.q_off : a.ny - 1;
        if (surf) base += (int64_t)a.q_off * sc;
        const int Qlo = pos0 * NG;
        for (int v = threadIdx.x; v < NP * SPAN; v += GB_THREADS) {
            const int P = v / SPAN, Q = Qlo + (v - (v / SPAN) * SPAN);
            const int p = P - a.vrows, q = Q - a.NQV;
            if (p < 0 || p >= a.nx || q < qlo || q > qhi) continue;
            const int l = P / NG, g = P - (P / NG) * NG;
            const int tq = Q + g, pos = tq / NG, w = tq - (tq / NG) * NG;   // pos - pos0 in [0, npos)
            base[(int64_t)p * sr + (int64_t)q * sc] = sl[((pos - pos0) * 32 + l) * SS + w * WS + band_gpos<NG>(g)];
        }
    }
}

template <int R, int LAM>
__host__ __device__ constexpr int adj_warp_floats() {
    return 2 * 32 * (R >> LAM) * (R >> LAM) + 2 * R;
}

template <int R, int LAM>
__global__ void __launch_bounds__(BAND_WARPS * 32, 6) chain_band_adj_kernel(BandAdjArgs a) {
    constexpr int S = 1 << LAM;
    constexpr int NG = R / S;
    constexpr int H = R / 2;
    constexpr int NH = NG / 2;
    constexpr int JOUT = R - 2;
    constexpr int SLOT = NG * NG;
    constexpr int NCH = SLOT >= 4 ? SLOT / 4 : 1;   // 16-byte chunks of a lane's slot
    extern __shared__ __align__(16) float adj_sm[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * BAND_WARPS + warp;
    const int64_t k0 = gw * a.ppw;
    if (k0 >= a.n_pairs) return;
    const int np = (int)min(a.ppw, a.n_pairs - k0);
    const int TperR = a.TperR;
    // per warp: two macro-steps of coefficient slots (lane-major, 16-byte
    // chunks rotated by lane against bank conflicts) and of the last row's Q
    float *ring = adj_sm + (size_t)warp * adj_warp_floats<R, LAM>();
    float *bqs = ring + 2 * 32 * SLOT;
    const float *bq = a.botq + gw * a.bq_stride;
    auto chunk = [&](int c) { return NCH >= 8 ? (c ^ (lane & 7)) : (NCH >= 2 ? (c ^ (lane & (NCH - 1))) : c); };
    auto lane_slot = [&](int buf) { return ring + ((size_t)buf * 32 + lane) * SLOT; };

    auto locate = [&](int64_t m, int &kl, int &pos) {
        const int64_t mm = m - lane;
        int64_t q = mm >= 0 ? mm / TperR : -((-mm + TperR - 1) / TperR);
        kl = (int)q;
        pos = (int)(mm - q * TperR);
    };
    auto slot_ptr = [&](int kk, int pp) -> const float * {
        if (kk < 0 || kk > np || (kk == np && pp != 0)) return nullptr;
        return a.band + (((k0 + kk) * TperR + pp) * 32 + lane) * (int64_t)SLOT;
    };
    // window w of macro-step m (slot src, null outside the chain) into buffer m & 1;
    // with window NG-1 also the last row's Q
    auto fetch = [&](int64_t m, const float *src, int w) {
        float *dst = lane_slot((int)(m & 1));
        if constexpr (NG == 8) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float *dd = dst + 4 * chunk(2 * w + h);
                if (src) cp_async<16>(dd, src + w * NG + 4 * h);
                else *reinterpret_cast<float4 *>(dd) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else if constexpr (NG == 4) {
            float *dd = dst + 4 * chunk(w);
            if (src) cp_async<16>(dd, src + w * NG);
            else *reinterpret_cast<float4 *>(dd) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            float *dd = dst + 2 * w;
            if (src) cp_async<8>(dd, src + w * NG);
            else *reinterpret_cast<float2 *>(dd) = make_float2(0.f, 0.f);
        }
        if (w == NG - 1 && lane == 31) {
            float *bd = bqs + (m & 1) * R;
#pragma unroll
            for (int h = 0; h < R / 4; ++h) cp_async<16>(bd + 4 * h, bq + m * R + 4 * h);
        }
    };
    auto read_window = [&](int buf, int w, float2 (&c)[NH]) {
        const float *sl = lane_slot(buf);
        float v[NG];
        if constexpr (NG == 8) {
            const float4 x0 = *reinterpret_cast<const float4 *>(sl + 4 * chunk(2 * w));
            const float4 x1 = *reinterpret_cast<const float4 *>(sl + 4 * chunk(2 * w + 1));
            v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
            v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        } else if constexpr (NG == 4) {
            const float4 x0 = *reinterpret_cast<const float4 *>(sl + 4 * chunk(w));
            v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
        } else {
            const float2 x0 = *reinterpret_cast<const float2 *>(sl + 2 * w);
            v[0] = x0.x; v[1] = x0.y;
        }
#pragma unroll
        for (int g = 0; g < NH; ++g) c[g] = make_float2(v[2 * g], v[2 * g + 1]);   // groups g, g + NH
    };

    // forward state as (K, -Q): undoing a step then needs no negation
    float2 KP[H], QN[H], A[H], V[H];
    float2 gN[NH], gO[NH];
    // coefficients of the window processed before (the next one in forward
    // order): a row's coefficient one forward step later comes from these or
    // from the current window's
    float2 CNP[NH];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        A[i] = make_float2(0.f, 0.f); V[i] = A[i];
        KP[i] = make_float2(1.f, 1.f); QN[i] = A[i];
    }
#pragma unroll
    for (int g = 0; g < NH; ++g) { gN[g] = make_float2(0.f, 0.f); gO[g] = gN[g]; CNP[g] = gN[g]; }

    const int64_t mlast = (int64_t)np * TperR + 31;
    int kl, pos;   // this lane's pair and position at macro-step m, tracked backwards
    locate(mlast, kl, pos);
    {
        const float *s0 = slot_ptr(kl, pos);
#pragma unroll
        for (int w = NG - 1; w >= 0; --w) {
            fetch(mlast, s0, w);
            cp_commit();
        }
    }

    for (int64_t m = mlast; m >= 0; --m) {
        if (m != mlast && --pos < 0) {
            pos = TperR - 1;
            --kl;
        }
        const bool trans = (pos == 0);
        const float *sprev = nullptr;
        if (m >= 1) sprev = pos > 0 ? slot_ptr(kl, pos - 1) : slot_ptr(kl - 1, TperR - 1);
        if ((m + 1) % BAND_CK == 0 || m == mlast) {
            // the forward's state after macro-step m
            const float4 *ck = reinterpret_cast<const float4 *>(
                a.ckpt + ((gw * a.nck + m / BAND_CK) * 32 + lane) * (int64_t)(2 * R));
#pragma unroll
            for (int i = 0; i < H; i += 2) {
                const float4 kk4 = ck[i / 2], qq4 = ck[H / 2 + i / 2];
                KP[i] = make_float2(kk4.x, kk4.y); KP[i + 1] = make_float2(kk4.z, kk4.w);
                QN[i] = make_float2(-qq4.x, -qq4.y); QN[i + 1] = make_float2(-qq4.z, -qq4.w);
            }
        }
        const bool cur_ok = kl >= 0 && kl < np, prev_ok = kl >= 1 && kl <= np;
        // the lane's slot rows in the dk/dc band: this pair's position, and at
        // position 0 also the previous pair's tail slot (its cells with w < g)
        float *gs_cur = cur_ok ? a.gband + (((k0 + kl) * (TperR + 1) + pos) * 32 + lane) * (int64_t)SLOT : nullptr;
        float *gs_prev = (trans && prev_ok)
                             ? a.gband + (((k0 + kl - 1) * (TperR + 1) + TperR) * 32 + lane) * (int64_t)SLOT
                             : nullptr;
        // rows turning over in this macro-step leave pair kl - 1 in reverse;
        // lane 31 seeds that pair's incoming gradient at its corner
        float gseed = 0.f;
        const bool has_prev = trans && prev_ok;
        float exK[R];   // their K when they left it (rows 0 .. R-1)
#pragma unroll
        for (int i = 0; i < R; ++i) exK[i] = 1.f;
        if (has_prev) {
            const float4 *ex = reinterpret_cast<const float4 *>(a.exitk + ((k0 + kl - 1) * 32 + lane) * (int64_t)R);
#pragma unroll
            for (int i = 0; i < R / 4; ++i) {
                const float4 v = ex[i];
                exK[4 * i] = v.x; exK[4 * i + 1] = v.y; exK[4 * i + 2] = v.z; exK[4 * i + 3] = v.w;
            }
            if (lane == 31) {
                // a symmetric Gram's pair (i, j), i < j, stands for (j, i) too
                const PairRef pr = pair_ref(a.src, k0 + kl - 1);
                gseed = a.gout[pr.out0] + (pr.out1 >= 0 ? a.gout[pr.out1] : 0.f);
            }
        }
        const int buf = (int)(m & 1);

        // a runtime loop over the windows keeps the body within the instruction cache
#pragma unroll 1
        for (int w = NG - 1; w >= 0; --w) {
            if (m >= 1) fetch(m - 1, sprev, w);
            cp_commit();
            cp_wait<NG - 1>();   // window w - 1 of this macro-step (w = 0: window NG-1 of the one before)
            float2 CN[NH], CO[NH];
            read_window(buf, w, CN);
            if (w > 0) read_window(buf, w - 1, CO);
            else read_window(buf ^ 1, NG - 1, CO);
            const int tw = has_prev ? w : -1;   // group whose rows turn over in this window

#pragma unroll
            for (int jj = S - 1; jj >= 0; --jj) {
                const int j = w * S + jj;
                const float qbot = bqs[buf * R + j];          // lane 31: its last row's Q before the step
                const float vH = V[0].y;
                float vd = __shfl_down_sync(FULL, V[0].x, 1);
                if (lane == 31) vd = (has_prev && j == JOUT) ? gseed : 0.f;
                // packed rows (H-1, R-1) first: their K before the step is the
                // row above packed row 0's
                constexpr int gH = (H - 1) / S, sH = (H - 1) % S;
                const bool hx = jj == sH && tw == gH, hy = jj == sH && tw == gH + NH;
                float2 KlH = add2(KP[H - 1], QN[H - 1]);
                float2 KpH = make_float2(hx ? exK[H - 1] : KlH.x, hy ? exK[R - 1] : KlH.y);
                KlH = make_float2(hx ? 1.f : KlH.x, hy ? 1.f : KlH.y);
                float pKs = __shfl_up_sync(FULL, KpH.y, 1);
                if (lane == 0) pKs = 1.f;
                float2 kprev = make_float2(pKs, KpH.x);
                float2 t0 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    const int g1 = i / S, s1 = i % S;
                    const bool px = jj == s1 && tw == g1, py = jj == s1 && tw == g1 + NH;
                    float2 Kl, Kp;
                    if (i == H - 1) {
                        Kl = KlH;
                        Kp = KpH;
                    } else {
                        Kl = add2(KP[i], QN[i]);
                        Kp = Kl;
                        if (jj == s1) {
                            Kp = make_float2(px ? exK[i] : Kl.x, py ? exK[i + H] : Kl.y);
                            Kl = make_float2(px ? 1.f : Kl.x, py ? 1.f : Kl.y);
                        }
                    }
                    const float2 sum = add2(Kl, kprev);
                    const float2 c = (jj >= s1) ? CN[g1] : CO[g1];
                    const float2 tq = fma2(c, sum, QN[i]);   // -Q before the step of the rows above
                    if (i == 0) t0 = tq;
                    else QN[i - 1] = tq;
                    KP[i] = Kp;
                    kprev = Kp;
                    const float2 vb = (i < H - 1) ? V[i < H - 1 ? i + 1 : 0] : make_float2(vH, vd);
                    // the row's coefficient one forward step later
                    const float2 cp = (jj < S - 1) ? ((jj + 1 >= s1) ? CN[g1] : CO[g1])
                                                   : (s1 == 0 ? CNP[g1] : CN[g1]);
                    const float2 P = fma2(cp, A[i], vb);
                    float2 An = add2(A[i], P);
                    V[i] = fma2(c, An, P);
                    if (jj >= s1) gN[g1] = fma2(An, sum, gN[g1]);
                    else gO[g1] = fma2(An, sum, gO[g1]);
                    // in reverse the row enters its previous pair: A(., Nj+1) = 0
                    if (jj == s1) An = make_float2(px ? 0.f : An.x, py ? 0.f : An.y);
                    A[i] = An;
                }
                float qd = __shfl_down_sync(FULL, t0.x, 1);
                if (lane == 31) qd = -qbot;
                QN[H - 1] = make_float2(t0.y, qd);
            }
            // window w's cells are complete: (P, Q) = (lane*NG + g, pos*NG + w - g),
            // in the order of the band's groups (g, g + NH side by side): one
            // vector store of the window row per slot
            if (a.src.scheme != SIGK_SCHEME_EXPLICIT) {   // dk/dc' -> dk/dc of the cell's coefficient
#pragma unroll
                for (int g = 0; g < NH; ++g) {
                    gN[g].x *= scheme_dcoef(CN[g].x, a.src.scheme);
                    gN[g].y *= scheme_dcoef(CN[g].y, a.src.scheme);
                }
            }
            if (gs_cur) store_window<NG>(gs_cur + w * NG, gN);
            if (gs_prev) store_window<NG>(gs_prev + w * NG, gN);
#pragma unroll
            for (int g = 0; g < NH; ++g) { gN[g] = gO[g]; gO[g] = make_float2(0.f, 0.f); CNP[g] = CN[g]; }
        }
    }
    cp_wait<0>();
}

// Real (unpadded) increments of paths: inc[(path * (L - 1) + p) * d + c].
__global__ void band_inc_kernel(const float *pts, int64_t npaths, int64_t L, int64_t d, float *inc) {
    const int64_t total = npaths * (L - 1) * d;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = v % d, row = v / d;
        const int64_t path = row / (L - 1), p = row - path * (L - 1);
        const float *x = pts + (path * L + p) * d + c;
        inc[v] = x[d] - x[0];
    }
}

// The chain rule through G(p, q) = <dx_p, dy_q>: C (+)= G B per batch, where
// G is dk/dc read straight from the adjoint's band layout (pair k's value at
// row-role increment p, column-role increment q sits in slot (k, pos, lane)
// at [w][gpos(g)] with P = p + vrows = lane NG + g, Q = q + NQV = pos NG + w - g).
// Not trans: C rows are the row role's increments (all row paths), the sum
// runs over the column role's; trans: the other way round.  Output tiles are
// 128 band coordinates (P, or Q when trans) of one output path by 32
// channels; reduction slices are 32 band coordinates of one reduction path.
// A slice's slots are staged whole (contiguous 16-byte loads), then
// transposed into the tile in shared memory; virtual rows and columns (the
// band's padding) read as zero.  4 x 4 outputs per thread; long reductions
// are split across blocks whose partial tiles a second kernel sums in order.
struct GemmArgs {
    const float *G;          // dense dk/dc (the tensor-core contraction only)
    int64_t g_ld;
    const float *Bm;
    int64_t b_bstride;
    float *C;
    int64_t c_bstride;
    int64_t M, K;            // output rows, reduction length (real increments)
    int N, trans, ksplit;    // ksplit > 1 (one batch only): block ks writes its partial
    float *partial;          // tile to partial[ks][M][N], summed by band_split_sum_kernel
    int64_t tri_rb, tri_cb;  // symmetric Gram: only pairs i <= j are stored (tensor-core path)
    const float *band;
    int mode;                // PM_PAIRS: batch b is pair b; PM_GRAM / PM_GRAM_SYM: one batch
    int64_t nb, a0, kbase;   // Gram: column paths, the launch's first row path, its first pair
    int64_t nA, nB;          // row / column paths of a batch (1 and 1 for pairs)
    int TperR1, vrows, NQV, nx, ny;
};
constexpr int GEMM_MAX_SPLIT = 8;
constexpr int GT_M = 128, GT_K = 32, GT_N = 32;

// the launch-local pair of row path ia and column path jb (-1: none stored,
// below a symmetric Gram's diagonal)
__device__ __forceinline__ int64_t gemm_pair(const GemmArgs &a, int64_t b, int64_t ia, int64_t jb) {
    if (a.mode == PM_PAIRS) return b;
    if (a.mode == PM_GRAM) return (a.a0 + ia) * a.nb + jb - a.kbase;
    if (ia > jb) return -1;
    return ia * a.nb - ia * (ia - 1) / 2 + (jb - ia) - a.kbase;
}

template <int NG>
__global__ void __launch_bounds__(256) band_gemm_kernel(GemmArgs a) {
    constexpr int SLOT = NG * NG;
    constexpr int BH = 32 * NG;                                           // band rows of a path
    constexpr int TL0 = (BH < GT_M ? BH : GT_M) / NG, TP0 = GT_K / NG + 1;   // staged lanes, positions
    constexpr int TL1 = GT_K / NG, TP1 = GT_M / NG + 1;                      // (trans)
    constexpr int ST0 = TL0 * TP0 * SLOT, ST1 = TL1 * TP1 * SLOT;
    constexpr int STF = ST0 > ST1 ? ST0 : ST1;
    constexpr int SV = (STF / 4 + 255) / 256;   // staged float4s per thread
    __shared__ __align__(16) float Gs[GT_K][GT_M + 4];
    __shared__ __align__(16) float Bs[GT_K][GT_N];
    __shared__ __align__(16) float St[STF];
    const bool tr = a.trans != 0;
    const int64_t b = blockIdx.z / a.ksplit;
    const int ks = blockIdx.z - (int)b * a.ksplit;
    const float *Bm = a.Bm + b * a.b_bstride;
    float *C = a.C + b * a.c_bstride;
    const int NQ = (a.TperR1 - 1) * NG;   // band columns of a path
    const int ocoords = tr ? NQ : BH;     // output band coordinates of a path
    const int tpp = (ocoords + GT_M - 1) / GT_M;
    const int64_t opath = blockIdx.x / tpp;
    const int o0 = (int)(blockIdx.x - opath * tpp) * GT_M;
    const int n0 = blockIdx.y * GT_N;
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
    // the reduction: paths [rlo, rhi) (a symmetric Gram stores pairs i <= j
    // only), each in spp slices of 32 band coordinates
    const int rcoords = tr ? BH : NQ;
    const int spp = (rcoords + GT_K - 1) / GT_K;
    int64_t rlo = 0, rhi = tr ? a.nA : a.nB;
    if (a.mode == PM_GRAM_SYM) {
        if (tr) rhi = opath + 1; else rlo = opath;
    }
    const int64_t total = (rhi - rlo) * spp;
    const int64_t s_lo = total * ks / a.ksplit, s_hi = total * (ks + 1) / a.ksplit;
    const int TL = tr ? TL1 : TL0, TP = tr ? TP1 : TP0;
    const int SN = TL * TP * SLOT / 4;   // float4s staged a slice
    const int nrr = tr ? a.nx : a.ny;    // real increments of the reduction role
    const int nro = tr ? a.ny : a.nx;    // and of the output role
    const int vro = tr ? a.NQV : a.vrows, vrr = tr ? a.vrows : a.NQV;

    float4 sv[SV];
    float br[4];
    int c0n = 0;
    // slice sidx into registers: its slots (not trans: lanes o0/NG + [0, TL0),
    // positions c0/NG + [0, TP0); trans: lanes c0/NG + [0, TL1), positions
    // o0/NG + [0, TP1); positions past the pair's last slot read as zero) and
    // the reduction role's 32 increments of 32 channels
    auto load = [&](int64_t sidx) {
        const int64_t rp = rlo + sidx / spp;
        const int c0 = (int)(sidx - (rp - rlo) * spp) * GT_K;
        const int64_t k = tr ? gemm_pair(a, b, rp, opath) : gemm_pair(a, b, opath, rp);
        const int l0 = (tr ? c0 : o0) / NG, p0 = (tr ? o0 : c0) / NG;
#pragma unroll
        for (int i = 0; i < SV; ++i) {
            const int u = threadIdx.x + 256 * i;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (u < SN && k >= 0) {
                const int sl = u / (SLOT / 4), e = u - sl * (SLOT / 4);
                const int pr = sl / TL, lr = sl - pr * TL;
                const int pos = p0 + pr;
                if (pos < a.TperR1)
                    v = __ldg(reinterpret_cast<const float4 *>(
                                  a.band + ((k * a.TperR1 + pos) * 32 + l0 + lr) * (int64_t)SLOT) + e);
            }
            sv[i] = v;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int v = threadIdx.x + 256 * i;
            const int kk = v / GT_N, nn = v % GT_N;
            const int real = c0 + kk - vrr;
            const int n = n0 + nn;
            br[i] = (real >= 0 && real < nrr && n < a.N && k >= 0) ? Bm[(rp * nrr + real) * a.N + n] : 0.f;
        }
        c0n = c0;
    };
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) acc[i][jx] = 0.f;
    if (s_lo < s_hi) load(s_lo);
    for (int64_t sidx = s_lo; sidx < s_hi; ++sidx) {
        const int c0 = c0n;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SV; ++i) {
            const int u = threadIdx.x + 256 * i;
            if (u < SN) reinterpret_cast<float4 *>(St)[u] = sv[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int v = threadIdx.x + 256 * i;
            Bs[v / GT_N][v % GT_N] = br[i];
        }
        __syncthreads();
        // Gs[kk][rr]: output coordinate o0 + rr, reduction coordinate c0 + kk;
        // virtual rows and columns of the reduction role read as zero
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int v = threadIdx.x + 256 * i;
            const int rr = v % GT_M, kk = v / GT_M;
            const int Prel = tr ? kk : rr, Qrel = tr ? rr : kk;
            const int lr = Prel / NG, g = Prel % NG;
            const int t = Qrel + g, pr = t / NG, w = t % NG;
            const int real = c0 + kk - vrr;
            const bool ok = real >= 0 && real < nrr && (tr || o0 + rr < BH);
            Gs[kk][rr] = ok ? St[(pr * TL + lr) * SLOT + w * NG + band_gpos<NG>(g)] : 0.f;
        }
        if (sidx + 1 < s_hi) load(sidx + 1);
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GT_K; ++kk) {
            const float4 gv = *reinterpret_cast<const float4 *>(&Gs[kk][4 * ty]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
            const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
            const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jx = 0; jx < 4; ++jx) acc[i][jx] = fmaf(gg[i], bb[jx], acc[i][jx]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int oc = o0 + 4 * ty + i;
        const int real = oc - vro;
        if (oc >= ocoords || real < 0 || real >= nro) continue;
        const int64_t r = opath * nro + real;
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) {
            const int n = n0 + 4 * tx + jx;
            if (n >= a.N) continue;
            if (a.ksplit > 1) a.partial[((int64_t)ks * a.M + r) * a.N + n] = acc[i][jx];
            else C[r * a.N + n] = acc[i][jx];
        }
    }
}

// ---- the RBF lift's chain rule (Sec. 2.2) ---------------------------------
// With c(p, q) = 1/2 4^-lambda (k(p+1,q+1) - k(p+1,q) - k(p,q+1) + k(p,q)),
// k(i, j) = kappa(x_i, y_j) = exp(-|x_i - y_j|^2 / (2 sigma^2)), the adjoint's
// dk/dc = Gbar gives dL/dk(i, j) = 1/2 4^-lambda W(i, j) with the second
// difference W(i, j) = Gbar(i-1,j-1) - Gbar(i-1,j) - Gbar(i,j-1) + Gbar(i,j)
// (Gbar zero outside the grid), and dk/dx_i = k (y_j - x_i) / sigma^2.  So
// with Wt = 1/2 4^-lambda W k over the points of every pair,
//   dL/dx_i = (sum_j Wt(i,j) y_j - x_i sum_j Wt(i,j)) / sigma^2
// and the mirror for y: a dense contraction of Wt with the points plus the
// row and column sums of Wt.

// C (+)= G B per batch for a dense G read as G[r * ld + k] (or G[k * ld + r]
// when trans).  128 x 32 output tiles, 32-deep K slices staged in shared
// memory (the next slice is loaded into registers while the current one is
// used), 4 x 4 outputs per thread; long K ranges split across blocks whose
// partial tiles band_split_sum_kernel adds in order.  A symmetric Gram's Wt
// holds blocks i <= j only (tri_rb x tri_cb blocks): the K slices of blocks
// below the diagonal are skipped.
struct DenseGemmArgs {
    const float *G;
    int64_t g_ld, g_bstride;
    const float *Bm;
    int64_t b_bstride;
    float *C;
    int64_t c_bstride;
    int64_t M, K;
    int N, trans, ksplit;
    float *partial;
    int64_t tri_rb, tri_cb;
};

__global__ void __launch_bounds__(256) dense_gemm_kernel(DenseGemmArgs a) {
    __shared__ __align__(16) float Gs[GT_K][GT_M + 4];
    __shared__ __align__(16) float Bs[GT_K][GT_N];
    const int64_t b = blockIdx.z / a.ksplit;
    const int ks = blockIdx.z - (int)b * a.ksplit;
    const float *G = a.G + b * a.g_bstride;
    const float *Bm = a.Bm + b * a.b_bstride;
    float *C = a.C + b * a.c_bstride;
    const int64_t r0 = (int64_t)blockIdx.x * GT_M;
    const int n0 = blockIdx.y * GT_N;
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
    // this block's K range, in whole slices
    int64_t kmin = 0, kmax = a.K;
    if (a.tri_rb > 0) {
        if (!a.trans) kmin = (r0 / a.tri_rb) * a.tri_cb;   // rows of block i: columns of blocks j >= i
        else {                                           // columns of block j: rows of blocks i <= j
            const int64_t rl = (r0 + GT_M - 1 < a.M ? r0 + GT_M - 1 : a.M - 1);
            kmax = (rl / a.tri_cb + 1) * a.tri_rb;
            if (kmax > a.K) kmax = a.K;
        }
    }
    const int64_t sl0 = kmin / GT_K, nslice = (kmax + GT_K - 1) / GT_K - sl0;
    const int64_t s_lo = sl0 + nslice * ks / a.ksplit, s_hi = sl0 + nslice * (ks + 1) / a.ksplit;
    float gr[16], br[4];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int v = threadIdx.x + 256 * i;
            int rr, kk;
            if (!a.trans) { rr = v / GT_K; kk = v % GT_K; } else { kk = v / GT_M; rr = v % GT_M; }
            const int64_t r = r0 + rr, k = k0 + kk;
            gr[i] = (r < a.M && k < a.K) ? (a.trans ? G[k * a.g_ld + r] : G[r * a.g_ld + k]) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int v = threadIdx.x + 256 * i;
            const int kk = v / GT_N, nn = v % GT_N;
            const int64_t k = k0 + kk;
            const int n = n0 + nn;
            br[i] = (k < a.K && n < a.N) ? Bm[k * a.N + n] : 0.f;
        }
    };
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) acc[i][jx] = 0.f;
    if (s_lo < s_hi) load(s_lo * GT_K);
    for (int64_t sl = s_lo; sl < s_hi; ++sl) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int v = threadIdx.x + 256 * i;
            if (!a.trans) Gs[v % GT_K][v / GT_K] = gr[i];
            else Gs[v / GT_M][v % GT_M] = gr[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int v = threadIdx.x + 256 * i;
            Bs[v / GT_N][v % GT_N] = br[i];
        }
        __syncthreads();
        if (sl + 1 < s_hi) load((sl + 1) * GT_K);
#pragma unroll 8
        for (int kk = 0; kk < GT_K; ++kk) {
            const float4 g = *reinterpret_cast<const float4 *>(&Gs[kk][4 * ty]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
            const float gg[4] = {g.x, g.y, g.z, g.w};
            const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jx = 0; jx < 4; ++jx) acc[i][jx] = fmaf(gg[i], bb[jx], acc[i][jx]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + 4 * ty + i;
        if (r >= a.M) continue;
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) {
            const int n = n0 + 4 * tx + jx;
            if (n >= a.N) continue;
            if (a.ksplit > 1) a.partial[((int64_t)ks * a.M + r) * a.N + n] = acc[i][jx];
            else C[r * a.N + n] = acc[i][jx];
        }
    }
}

// C = (add ? C : 0) + sum over the splits, in split order (deterministic).
__global__ void band_split_sum_kernel(const float *partial, int ksplit, int64_t MN, int add, float *C) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < MN; v += (int64_t)gridDim.x * blockDim.x) {
        float acc = add ? C[v] : 0.f;
        for (int s = 0; s < ksplit; ++s) acc += partial[s * MN + v];
        C[v] = acc;
    }
}

// Point gradients from increment gradients: x_p enters dx_{p-1} (+) and dx_p
// (-), so dX[path][p] = scale (dinc[p-1] - dinc[p]) (terms outside 0..L-2
// absent).  Overwrites dpts, or adds to it (add).
__global__ void band_points_kernel(const float *dinc, int64_t npaths, int64_t L, int64_t d, float scale,
                                   int add, float *dpts) {
    const int64_t total = npaths * L * d;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = v % d, row = v / d;
        const int64_t path = row / L, p = row - path * L;
        const float *di = dinc + path * (L - 1) * d + c;
        const float lo = p >= 1 ? di[(p - 1) * d] : 0.f;
        const float hi = p < L - 1 ? di[p * d] : 0.f;
        const float g = scale * (lo - hi);
        dpts[v] = add ? dpts[v] + g : g;
    }
}


// Wt of every pair's (nx+1) x (ny+1) points (see the RBF chain rule above)
// and its row and column sums.  Units are (pair, 128 x 32 point tile); a
// block stages the tile's points channel-major (32 channels a pass) and the
// 129 x 33 values of dk/dc around it from the band layout; thread t owns
// points rows 4 (t/8) .. +3 and columns 4 (t%8) .. +3 of the tile.
struct RbfWtArgs {
    PairSrc src;             // oriented: rows refine A
    const float *gband;      // dk/dc in the band layout (TperR1 slots per pair)
    float *wt;               // Gram: [row path ia][i] x [column path jb][j], ld = ldw; pairs: [k][i][j]
    float *rsum, *csum;      // sums over j / over i (zeroed before)
    int64_t n_pairs, ldw, a0;
    int TperR1, vrows, NQV, tiles_i, tiles_j;
    float s, scale;          // 1/(2 sigma^2), 1/2 4^-lambda
};
constexpr int RW_TI = 128, RW_TJ = 32, RW_CH = 32;

template <int NG>
__global__ void __launch_bounds__(256) rbf_wt_kernel(RbfWtArgs a) {
    constexpr int SLOT = NG * NG;
    // the band slots around a tile: lanes (rows) and positions (columns)
    constexpr int SL = RW_TI / NG + 1 < 32 ? RW_TI / NG + 1 : 32, SP = RW_TJ / NG + 2;
    // the points (channel loop) and the staged slots (before it) share memory
    constexpr int PTS = RW_CH * RW_TI + RW_CH * (RW_TJ + 1), STG = SL * SP * SLOT;
    __shared__ __align__(16) float pool[PTS > STG ? PTS : STG];
    float (*xs)[RW_TI] = reinterpret_cast<float (*)[RW_TI]>(pool);
    float (*ys)[RW_TJ + 1] = reinterpret_cast<float (*)[RW_TJ + 1]>(pool + RW_CH * RW_TI);
    __shared__ float gs[RW_TI + 1][RW_TJ + 2];
    const int tid = threadIdx.x, lane = tid & 31;
    const int r = (tid >> 3) * 4, c0 = (tid & 7) * 4;
    const int64_t d = a.src.d;
    const bool gram = a.src.mode != PM_PAIRS;
    const int per = a.tiles_i * a.tiles_j;
    for (int64_t u = blockIdx.x; u < a.n_pairs * per; u += gridDim.x) {
        const int64_t k = u / per;
        const int t = (int)(u - k * per);
        const int i0 = (t / a.tiles_j) * RW_TI, j0 = (t % a.tiles_j) * RW_TJ;
        const PairRef pr = pair_ref(a.src, k);
        const int nx = (int)pr.la - 1, ny = (int)pr.lb - 1;   // coarse rows / columns; nx + 1 points
        if (i0 > nx || j0 > ny) continue;   // block-uniform
        const float *xp = (const float *)a.src.A + pr.a_row0 * d;
        const float *yp = (const float *)a.src.B + pr.b_row0 * d;
        __syncthreads();
        // the slots holding dk/dc at (p, q) = (i0 - 1 + pi, j0 - 1 + qj): lanes
        // from l0, positions from s0 (for a position, the lanes are one
        // contiguous run), staged with 16-byte loads; then the tile, zero
        // outside the grid
        const int Pf = i0 - 1 + a.vrows, Qf = j0 - 1 + a.NQV;
        const int l0 = (Pf < 0 ? 0 : Pf) / NG, s0 = (Qf < 0 ? 0 : Qf) / NG;
        for (int v = tid; v < STG / 4; v += 256) {
            const int sl = v / (SLOT / 4), e = v - sl * (SLOT / 4);
            const int pr = sl / SL, lr = sl - pr * SL;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l0 + lr < 32 && s0 + pr < a.TperR1)
                x = __ldg(reinterpret_cast<const float4 *>(a.gband + ((k * a.TperR1 + s0 + pr) * 32 + l0 + lr) *
                                                                        (int64_t)SLOT) + e);
            reinterpret_cast<float4 *>(pool)[v] = x;
        }
        __syncthreads();
        for (int v = tid; v < (RW_TI + 1) * (RW_TJ + 1); v += 256) {
            const int pi = v / (RW_TJ + 1), qj = v - pi * (RW_TJ + 1);
            const int pp = i0 - 1 + pi, qq = j0 - 1 + qj;
            float gv = 0.f;
            if (pp >= 0 && pp < nx && qq >= 0 && qq < ny) {
                const int P = pp + a.vrows, Q = qq + a.NQV;
                const int l = P / NG, g = P % NG, tq = Q + g;
                gv = pool[((tq / NG - s0) * SL + l - l0) * SLOT + (tq % NG) * NG + band_gpos<NG>(g)];
            }
            gs[pi][qj] = gv;
        }
        // |x_i - y_j|^2 = |x_i|^2 + |y_j|^2 - 2 <x_i, y_j>: one FMA a pair and
        // channel (only kappa itself is needed here, so the cancellation near
        // x_i = y_j costs an absolute error of about FP32 epsilon times |x|^2)
        float xy[4][4], xx[4], yy[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xx[i] = 0.f;
            yy[i] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) xy[i][j] = 0.f;
        }
        for (int64_t cb = 0; cb < d; cb += RW_CH) {
            const int nc = d - cb < RW_CH ? (int)(d - cb) : RW_CH;
            __syncthreads();
            // consecutive threads take consecutive channels of a point (the
            // full-width passes without a division)
            for (int v = tid; v < nc * RW_TI; v += 256) {
                const int i = nc == RW_CH ? v >> 5 : v / nc, c = nc == RW_CH ? v & 31 : v - i * nc;
                xs[c][i] = i0 + i <= nx ? xp[(int64_t)(i0 + i) * d + cb + c] : 0.f;
            }
            for (int v = tid; v < nc * RW_TJ; v += 256) {
                const int j = nc == RW_CH ? v >> 5 : v / nc, c = nc == RW_CH ? v & 31 : v - j * nc;
                ys[c][j] = j0 + j <= ny ? yp[(int64_t)(j0 + j) * d + cb + c] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int c = 0; c < nc; ++c) {
                float xv[4], yv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = xs[c][r + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) yv[j] = ys[c][c0 + j];
#pragma unroll
                for (int j = 0; j < 4; ++j) yy[j] = fmaf(yv[j], yv[j], yy[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    xx[i] = fmaf(xv[i], xv[i], xx[i]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) xy[i][j] = fmaf(xv[i], yv[j], xy[i][j]);
                }
            }
        }
        float rs[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t ia = gram ? pr.a_row0 / pr.la - a.a0 : k;
        const int64_t jb = gram ? pr.b_row0 / pr.lb : k;
        // a row's four columns leave as one 16-byte store where the rows are
        // 16-byte aligned and all four are real
        const bool vec = ((ny + 1) & 3) == 0 && j0 + c0 + 3 <= ny;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pi = r + i, ii = i0 + pi;
            if (ii > nx) continue;
            float wv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qj = c0 + j;
                const float W = gs[pi][qj] - gs[pi][qj + 1] - gs[pi + 1][qj] + gs[pi + 1][qj + 1];
                const float uu = fmaxf(xx[i] + yy[j] - 2.f * xy[i][j], 0.f);
                wv[j] = j0 + qj <= ny ? a.scale * W * __expf(-a.s * uu) : 0.f;
                rs[i] += wv[j];
                cs[j] += wv[j];
            }
            float *row = gram ? a.wt + (ia * (nx + 1) + ii) * a.ldw + jb * (ny + 1)
                              : a.wt + (k * (nx + 1) + ii) * (int64_t)(ny + 1);
            if (vec) {
                *reinterpret_cast<float4 *>(row + j0 + c0) = make_float4(wv[0], wv[1], wv[2], wv[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j0 + c0 + j <= ny) row[j0 + c0 + j] = wv[j];
            }
        }
        // row sums over the 8 threads of a row group, column sums over the
        // 4 row groups of the warp; then one atomic add per value
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            rs[i] += __shfl_xor_sync(FULL, rs[i], 1);
            rs[i] += __shfl_xor_sync(FULL, rs[i], 2);
            rs[i] += __shfl_xor_sync(FULL, rs[i], 4);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cs[j] += __shfl_xor_sync(FULL, cs[j], 8);
            cs[j] += __shfl_xor_sync(FULL, cs[j], 16);
        }
        if ((lane & 7) == 0)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i0 + r + i <= nx) atomicAdd(a.rsum + ia * (nx + 1) + i0 + r + i, rs[i]);
        if (lane < 8)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j0 + c0 + j <= ny) atomicAdd(a.csum + jb * (ny + 1) + j0 + c0 + j, cs[j]);
    }
}

// out[v] = (add ? out[v] : 0) + f (C1[v] - s1[row] P[v] (+ C2[v] - s2[row] P[v])),
// v = row d + channel: the points' gradients from the contraction and the
// sums (C2, s2: the column role of a symmetric Gram's same paths)
__global__ void rbf_points_kernel(const float *P, int64_t rows, int64_t d, const float *C1, const float *s1,
                                  const float *C2, const float *s2, float f, int add, float *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < rows * d;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = v / d;
        float g = C1[v] - s1[row] * P[v];
        if (C2) g += C2[v] - s2[row] * P[v];
        out[v] = add ? out[v] + f * g : f * g;
    }
}

}  // namespace

bool band_geometry(int64_t La, int64_t Lb, int lam, int rows_per_lane, BandPlan &p) {
    if (La < 2 || Lb < 2 || lam < 0 || lam > 3) return false;
    const int64_t S = 1LL << lam;
    const int64_t Ni = S * (La - 1), Nj = S * (Lb - 1);
    int R = 0;
    for (int r : {4, 8, 16})
        if ((rows_per_lane == 0 || rows_per_lane == r) && 32 * r >= Ni && band_has_instance(r, lam)) {
            R = r;
            break;
        }
    if (R == 0) return false;
    const int NG = R >> lam;
    const int64_t Tper = ((Nj + R - 1) / R) * R;
    if (Tper < 2 * R || Tper > (1 << 20)) return false;
    p.R = R;
    p.lam = lam;
    p.NG = NG;
    p.TperR = (int)(Tper / R);
    p.NQ = (int)(Tper / S);
    p.NQV = (int)((Tper - Nj) / S);
    p.vrows = (int)((32 * R - Ni) / S);
    p.slot_floats = (int64_t)32 * NG * NG;
    return true;
}

// workspace: a 256-byte header (the status word of bounded waits), then the band
int64_t band_bytes(const BandPlan &p, int64_t n_pairs) {
    return 256 + (int64_t)sizeof(float) * (n_pairs * p.TperR + 1) * p.slot_floats;
}

// The surface's band-layout values (TperR + 1 slots per pair) after the band:
// their float offset from the band's start, and the whole workspace.
int64_t band_surface_offset(const BandPlan &p, int64_t n_pairs) {
    return ((n_pairs * p.TperR + 1) * p.slot_floats + 63) / 64 * 64;
}
int64_t band_surface_bytes(const BandPlan &p, int64_t n_pairs) {
    return 256 + (int64_t)sizeof(float) *
                     (band_surface_offset(p, n_pairs) + n_pairs * (p.TperR + 1) * p.slot_floats);
}

namespace {
// The band coefficients: the FMA contraction, or on request (coef_path 3,
// d <= 64) the tcgen05 kernel.  The FMA kernel is the default: it runs two
// blocks per SM and overlaps staging with arithmetic, where the tensor-core
// kernel's one block per SM serialises staging, MMAs and the scattered band
// write-back (measured on the 128 x 128 MMD Gram, d = 32: 1.5 vs 4.8 ms).
// Band layout of the RBF-lifted coefficients (rbf.cuh): coarse cell (p, q) of
// pair k is the padded cell (P, Q) = (p + vrows, q + NQV), read by lane P / NG
// as group g = P % NG at the position pos and window w with pos NG + w = Q + g;
// pos = TperR is the pair's tail, in slot 0 of pair k + 1.
template <int NG>
struct BandRbfLayout {
    PairSrc src;
    float *band;
    int TperR, NQV, vrows;
    struct Geo {
        const float *rows, *cols;
        int nx, ny;
        int64_t k;
    };
    struct Row {
        int64_t lane_off;   // (lane) * NG^2 + band_gpos(g)
        int gr;             // group of the row within its lane
    };
    __device__ Geo geo(int64_t k) const {
        const PairRef pr = pair_ref(src, k);
        Geo g;
        g.rows = (const float *)src.A + pr.a_row0 * src.d;
        g.cols = (const float *)src.B + pr.b_row0 * src.d;
        g.nx = (int)pr.la - 1;
        g.ny = (int)pr.lb - 1;
        g.k = k;
        return g;
    }
    __device__ Row row(const Geo &, int p) const {
        const int P = p + vrows;
        Row r;
        r.gr = P % NG;
        r.lane_off = (int64_t)(P / NG) * (NG * NG) + band_gpos<NG>(r.gr);
        return r;
    }
    __device__ void store(const Geo &g, const Row &r, int q, float c) const {
        const int t = q + NQV + r.gr, pos = t / NG, w = t % NG;
        const int64_t slot = pos < TperR ? g.k * TperR + pos : (g.k + 1) * TperR;
        band[slot * (32 * NG * NG) + r.lane_off + w * NG] = c;
    }
};

template <int NG>
cudaError_t launch_band_rbf(const BandCoefArgs &c, int sms, cudaStream_t st) {
    BandRbfLayout<NG> lay;
    lay.src = c.src;
    lay.band = c.band;
    lay.TperR = c.TperR;
    lay.NQV = c.NQV;
    lay.vrows = c.vrows;
    const size_t bytes = sizeof(float) * (size_t)(c.n_pairs * c.TperR + 1) * 32 * NG * NG;
    return launch_rbf_coef<float>(lay, c.n_pairs, c.src.La - 1, c.src.Lb - 1, c.src.d, c.src.sigma,
                                  (double)c.scale, c.src.scheme, c.band, bytes, sms, st);
}

cudaError_t launch_band_coef(const BandCoefArgs &c, int NG, int sms, int *status, cudaStream_t st,
                             int coef_path) {
    if (c.src.kernel == SIGK_KERNEL_RBF) {
        if (NG == 8) return launch_band_rbf<8>(c, sms, st);
        if (NG == 4) return launch_band_rbf<4>(c, sms, st);
        return launch_band_rbf<2>(c, sms, st);
    }
    if (coef_path == 3 && c.src.d <= 64) {
        if (NG == 8) return launch_coef_tc5<8>(c, sms, status, st);
        if (NG == 4) return launch_coef_tc5<4>(c, sms, status, st);
        return launch_coef_tc5<2>(c, sms, status, st);
    }
    if (NG == 8) return launch_coef<8>(c, sms, st);
    if (NG == 4) return launch_coef<4>(c, sms, st);
    return launch_coef<2>(c, sms, st);
}
}  // namespace

cudaError_t launch_band_f32(const PairSrc &src, const BandPlan &p, int64_t n_pairs, float *out,
                            void *ws, cudaStream_t st, int coef_path, float *surf, int64_t s_pair,
                            int64_t s_a, int64_t s_b) {
    if (n_pairs <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int *status = (int *)ws;
    float *band = (float *)((unsigned char *)ws + 256);
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), st)) != cudaSuccess) return e;
    BandCoefArgs c;
    c.src = src;
    c.n_pairs = n_pairs;
    c.TperR = p.TperR;
    c.NQ = p.NQ;
    c.NQV = p.NQV;
    c.vrows = p.vrows;
    c.scale = 0.5f / (float)(1 << (2 * p.lam));
    c.band = band;
    if ((e = launch_band_coef(c, p.NG, sms, status, st, coef_path)) != cudaSuccess) return e;

    const int per_sm = band_occupancy_of(p.R, p.lam);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t warps = (int64_t)sms * per_sm * BAND_WARPS;
    BandArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.out = out;
    a.band = band;
    a.n_pairs = n_pairs;
    a.ppw = (n_pairs + warps - 1) / warps;
    a.TperR = p.TperR;
    // the surface's band-layout values follow the coefficient band in the workspace
    a.sband = surf ? band + band_surface_offset(p, n_pairs) : nullptr;
    const int64_t nwarps = (n_pairs + a.ppw - 1) / a.ppw;
    const int grid = (int)((nwarps + BAND_WARPS - 1) / BAND_WARPS);
    bool launched = false;
#define X(r, l, mb)                                                                  \
    if (p.R == r && p.lam == l) {                                                    \
        if (surf)                                                                    \
            chain_band_kernel<r, l, mb, false, true><<<grid, BAND_WARPS * 32, 0, st>>>(a); \
        else                                                                         \
            chain_band_kernel<r, l, mb, false><<<grid, BAND_WARPS * 32, 0, st>>>(a);       \
        launched = true;                                                             \
    }
    SIGK_BAND_CASES(X)
#undef X
    if (!launched) return cudaErrorInvalidValue;
    if ((e = cudaGetLastError()) != cudaSuccess || !surf) return e;
    return launch_surface_unpack(src, p, n_pairs, a.sband, surf, s_pair, s_a, s_b, st);
}

cudaError_t launch_surface_unpack(const PairSrc &src, const BandPlan &p, int64_t n_pairs, const float *sband,
                                  float *surf, int64_t s_pair, int64_t s_a, int64_t s_b, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // the surface from the band layout into [pair][L][M]
    BandGbarArgs gb;
    memset(&gb, 0, sizeof(gb));
    gb.src = src;
    gb.gband = sband;
    gb.gbar = surf;
    gb.n_pairs = n_pairs;
    gb.TperR = p.TperR;
    gb.NQV = p.NQV;
    gb.vrows = p.vrows;
    gb.nx = (int)(src.La - 1);
    gb.ny = (int)(src.Lb - 1);
    gb.s_pair = s_pair;
    gb.s_a = s_a;
    gb.s_b = s_b;
    gb.q_off = p.lam == 0 ? 1 : 0;
    const int64_t tasks = n_pairs * gb_groups(p.TperR, true, p.NG);
    const int ggrid = (int)(tasks < (int64_t)sms * 8 ? tasks : (int64_t)sms * 8);
    if (p.NG == 8) band_gbar_kernel<8><<<ggrid, GB_THREADS, 0, st>>>(gb);
    else if (p.NG == 4) band_gbar_kernel<4><<<ggrid, GB_THREADS, 0, st>>>(gb);
    else band_gbar_kernel<2><<<ggrid, GB_THREADS, 0, st>>>(gb);
    return cudaGetLastError();
}

}  // namespace sigk

// ---- the band backward -------------------------------------------------------

namespace sigk {

namespace {

template <int R, int LAM>
cudaError_t launch_adj(const BandAdjArgs &a, int64_t nwarps, cudaStream_t st) {
    const int smem = (int)sizeof(float) * BAND_WARPS * adj_warp_floats<R, LAM>();
    auto kern = chain_band_adj_kernel<R, LAM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (nwarps + BAND_WARPS - 1) / BAND_WARPS;
    kern<<<(int)grid, BAND_WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

int64_t up4(int64_t v) { return (v + 3) / 4 * 4; }

// Float counts of the backward's workspace regions for a launch of nbp pairs
// (Gram: whole rows of nb pairs).  Checkpoint and last-row regions are sized
// for any pairs-per-warp split (they are checked against the actual split at
// launch).
struct BwdRegions {
    int64_t band, gbar, ckpt, exitk, botq, incA, incB, dincA, dincB, part, gband, rsum;
    int64_t total() const {
        return band + gbar + ckpt + exitk + botq + incA + incB + dincA + dincB + part + gband + rsum;
    }
};

// dense: whether a Gram's dk/dc is unpacked into a dense matrix for the
// tensor-core contraction (coef_path 3); the FP32 contraction reads the band
bool bwd_dense_gbar(const PairSrc &src, int coef_path) {
    const bool gram = src.mode == PM_GRAM || src.mode == PM_GRAM_SYM;
    return gram && src.kernel == SIGK_KERNEL_LINEAR && coef_path == 3 && chain_gemm_tc5_ok(1, 1, (int)src.d);
}

BwdRegions bwd_regions(const PairSrc &src, const BandPlan &p, int64_t nbp, int coef_path) {
    const int64_t nx = src.La - 1, ny = src.Lb - 1, d = src.d;
    const bool sym = src.mode == PM_GRAM_SYM;
    const bool gram = src.mode == PM_GRAM || sym;
    const int64_t nA = sym ? src.nb : gram ? (nbp + src.nb - 1) / src.nb : nbp;
    const int64_t nB = gram ? src.nb : nbp;
    BwdRegions r;
    r.band = up4(band_bytes(p, nbp) / (int64_t)sizeof(float));
    r.gbar = bwd_dense_gbar(src, coef_path) ? up4(nA * nx * nB * ny) : 0;
    r.ckpt = ((nbp + 1) * ((2 * (int64_t)p.TperR + 32 + BAND_CK) / BAND_CK) + 1) * 32 * 2 * p.R;
    r.exitk = (nbp + 1) * 32 * (int64_t)p.R;
    r.botq = up4((nbp + 1) * ((2 * (int64_t)p.TperR + 32) * p.R + 4));
    r.incA = up4(nA * nx * d);
    r.incB = up4(nB * ny * d);
    r.dincA = r.incA;
    r.dincB = r.incB;
    // split-K partial tiles of the Gram's contractions
    r.part = gram ? up4((int64_t)GEMM_MAX_SPLIT * (nA * nx > nB * ny ? nA * nx : nB * ny) * d) : 0;
    r.rsum = 0;
    if (src.kernel == SIGK_KERNEL_RBF) {
        // the lift works on points: Wt of every pair (dense, in gbar), the
        // contractions' results (dinc), the row and column sums; no increments
        const int64_t px = nx + 1, py = ny + 1;
        r.gbar = up4(nA * px * nB * py);
        if (!gram) r.gbar = up4(nbp * px * py);
        r.incA = r.incB = 0;
        r.dincA = up4(nA * px * d);
        r.dincB = up4(nB * py * d);
        r.part = gram ? up4((int64_t)GEMM_MAX_SPLIT * (nA * px > nB * py ? nA * px : nB * py) * d) : 0;
        r.rsum = up4(nA * px) + up4(nB * py);
    }
    // the adjoint's dk/dc in the band layout: TperR + 1 slots per pair
    r.gband = up4(nbp * ((int64_t)p.TperR + 1) * 32 * p.NG * p.NG);
    return r;
}

}  // namespace

int64_t band_bwd_batch(const PairSrc &src, const BandPlan &p, int64_t n, int64_t cap_bytes,
                       int64_t &bytes, int coef_path) {
    if (src.mode == PM_GRAM_SYM) {   // one launch: every pair involves the same paths
        bytes = bwd_regions(src, p, n, coef_path).total() * (int64_t)sizeof(float);
        return n;
    }
    // whole Gram rows per launch: each launch owns its row paths' gradients
    const int64_t unit = src.mode == PM_GRAM ? src.nb : 1;
    int64_t units = (n + unit - 1) / unit;
    int64_t nb = n;
    bytes = bwd_regions(src, p, nb, coef_path).total() * (int64_t)sizeof(float);
    while (units > 1 && bytes > cap_bytes) {
        units = (units + 1) / 2;
        nb = units * unit < n ? units * unit : n;
        bytes = bwd_regions(src, p, nb, coef_path).total() * (int64_t)sizeof(float);
    }
    return nb;
}

// The RBF lift's chain rule for one launch of the band backward (pairs
// kbase .. kbase + m of the oriented src; Gram: row paths a0 .. a0 + nA
// against all nB column paths): Wt and its sums, the dense contractions
// CX = Wt Y and CY = Wt^T X, then the points' gradients.  dA is overwritten
// (or added to: add); dB likewise on the first launch and added to after.
cudaError_t rbf_chain_rule(const PairSrc &src, const BandPlan &p, int64_t m, int64_t a0, int64_t nA, int64_t nB,
                           int64_t kb, const float *gband, float *wt, float *CX, float *CY, float *rsum,
                           float *part, float *dA, float *dB, bool add, int sms, cudaStream_t st) {
    const bool sym = src.mode == PM_GRAM_SYM;
    const bool gram = src.mode == PM_GRAM || sym;
    const int64_t d = src.d, px = src.La, py = src.Lb;   // points per path
    const int64_t nrow = gram ? nA : m, ncol = gram ? nB : m;
    float *csum = rsum + up4(nrow * px);
    cudaError_t e;
    if ((e = cudaMemsetAsync(rsum, 0, sizeof(float) * (size_t)(up4(nrow * px) + ncol * py), st)) != cudaSuccess)
        return e;
    // a symmetric Gram stores pairs i <= j: the blocks below the diagonal stay zero
    if (sym && (e = cudaMemsetAsync(wt, 0, sizeof(float) * (size_t)(nA * px * nB * py), st)) != cudaSuccess)
        return e;
    RbfWtArgs w;
    w.src = src;
    w.gband = gband;
    w.wt = wt;
    w.rsum = rsum;
    w.csum = csum;
    w.n_pairs = m;
    w.ldw = gram ? nB * py : py;
    w.a0 = a0;
    w.TperR1 = p.TperR + 1;
    w.vrows = p.vrows;
    w.NQV = p.NQV;
    w.tiles_i = (int)((px + RW_TI - 1) / RW_TI);
    w.tiles_j = (int)((py + RW_TJ - 1) / RW_TJ);
    w.s = (float)(0.5 / (src.sigma * src.sigma));
    w.scale = 0.5f / (float)(1 << (2 * p.lam));
    int64_t grid = m * w.tiles_i * w.tiles_j;
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    if (p.NG == 8) rbf_wt_kernel<8><<<(int)grid, 256, 0, st>>>(w);
    else if (p.NG == 4) rbf_wt_kernel<4><<<(int)grid, 256, 0, st>>>(w);
    else rbf_wt_kernel<2><<<(int)grid, 256, 0, st>>>(w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the contractions
    const float *Apts = (const float *)src.A + (gram ? a0 : src.kbase) * px * d;
    const float *Bpts = sym ? (const float *)src.A : (const float *)src.B + (gram ? 0 : src.kbase) * py * d;
    DenseGemmArgs g1;
    memset(&g1, 0, sizeof(g1));
    g1.G = wt;
    g1.N = (int)d;
    DenseGemmArgs g2 = g1;
    g1.Bm = Bpts;
    g1.C = CX;
    g1.trans = 0;
    g2.Bm = Apts;
    g2.C = CY;
    g2.trans = 1;
    int64_t batches = 1;
    if (gram) {
        g1.g_ld = g2.g_ld = nB * py;
        g1.M = nA * px; g1.K = nB * py;
        g2.M = nB * py; g2.K = nA * px;
        g1.tri_rb = g2.tri_rb = sym ? px : 0;
        g1.tri_cb = g2.tri_cb = sym ? py : 0;
    } else {
        batches = m;
        g1.g_ld = g2.g_ld = py;
        g1.g_bstride = g2.g_bstride = px * py;
        g1.b_bstride = py * d; g2.b_bstride = px * d;
        g1.c_bstride = px * d; g2.c_bstride = py * d;
        g1.M = px; g1.K = py;
        g2.M = py; g2.K = px;
    }
    auto split = [&](const DenseGemmArgs &g) {
        if (!gram) return 1;
        const int64_t tiles = ((g.M + GT_M - 1) / GT_M) * ((d + GT_N - 1) / GT_N);
        int64_t ksp = (4 * (int64_t)sms + tiles - 1) / tiles;
        const int64_t nsl = (g.K + GT_K - 1) / GT_K;
        if (ksp > nsl / 4) ksp = nsl / 4;
        if (ksp > GEMM_MAX_SPLIT) ksp = GEMM_MAX_SPLIT;
        return (int)(ksp < 1 ? 1 : ksp);
    };
    g1.ksplit = split(g1);
    g2.ksplit = split(g2);
    g1.partial = g2.partial = part;
    const bool want_b = dB || sym;
    for (int pass = 0; pass < (want_b ? 2 : 1); ++pass) {
        const DenseGemmArgs &g = pass == 0 ? g1 : g2;
        const dim3 gd((unsigned)((g.M + GT_M - 1) / GT_M), (unsigned)((d + GT_N - 1) / GT_N),
                      (unsigned)(batches * g.ksplit));
        dense_gemm_kernel<<<gd, 256, 0, st>>>(g);
        if (g.ksplit > 1) band_split_sum_kernel<<<sms * 4, 256, 0, st>>>(part, g.ksplit, g.M * d, 0, g.C);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the points
    const float f = (float)(1.0 / (src.sigma * src.sigma));
    if (dA) {
        float *out = dA + (gram ? a0 : src.kbase) * px * d;
        rbf_points_kernel<<<sms * 4, 256, 0, st>>>(Apts, nrow * px, d, CX, rsum, sym ? CY : nullptr,
                                                   sym ? csum : nullptr, f, add ? 1 : 0, out);
    }
    if (dB && !sym) {
        float *out = dB + (gram ? 0 : src.kbase) * py * d;
        rbf_points_kernel<<<sms * 4, 256, 0, st>>>(Bpts, ncol * py, d, CY, csum, nullptr, nullptr, f,
                                                   (add || (gram && kb > 0)) ? 1 : 0, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_band_bwd_f32(const PairSrc &src0, const BandPlan &p, int64_t n, int64_t nbp,
                                const float *gout, float *dA, float *dB, void *ws, cudaStream_t st,
                                int coef_path, float *out, bool add) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int per_sm = band_occupancy_of(p.R, p.lam);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // symmetric Gram: pairs (i, j), i <= j, of one batch; dA gets the
    // derivative through both arguments (dB must be null)
    const bool sym = src0.mode == PM_GRAM_SYM;
    const bool gram = src0.mode == PM_GRAM || sym;
    if (sym && (dB || nbp != n)) return cudaErrorInvalidValue;
    const int64_t nx = src0.La - 1, ny = src0.Lb - 1, d = src0.d;
    const float scale = 0.5f / (float)(1 << (2 * p.lam));
    const BwdRegions rg = bwd_regions(src0, p, nbp, coef_path);
    float *w = (float *)ws;
    int *status = (int *)ws;
    float *band = w + 64;   // after the 256-byte status header
    float *gbar = w + rg.band;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), st)) != cudaSuccess) return e;
    float *ckpt = gbar + rg.gbar;
    float *exitk = ckpt + rg.ckpt;
    float *botq = exitk + rg.exitk;
    float *incA = botq + rg.botq;
    float *incB = incA + rg.incA;
    float *dincA = incB + rg.incB;
    float *dincB = dincA + rg.dincA;
    float *part = dincB + rg.dincB;
    float *gband = part + rg.part;
    float *rsum = gband + rg.gband;   // the RBF lift's row sums, then its column sums
    const bool rbf = src0.kernel == SIGK_KERNEL_RBF;
    const int64_t nBall = gram ? src0.nb : 0;
    if (gram && !rbf) {
        // every column path is used by every launch: increments once, gradients summed
        band_inc_kernel<<<sms * 4, 256, 0, st>>>((const float *)src0.B, nBall, src0.Lb, d, incB);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int64_t kb = 0; kb < n; kb += nbp) {
        const int64_t m = n - kb < nbp ? n - kb : nbp;
        PairSrc src = src0;
        src.kbase = src0.kbase + kb;
        const int64_t a0 = sym ? 0 : gram ? src.kbase / src0.nb : src.kbase;   // first row path
        const int64_t nA = sym ? src0.nb : gram ? m / src0.nb : m;
        // 1. coefficients
        BandCoefArgs c;
        c.src = src;
        c.n_pairs = m;
        c.TperR = p.TperR;
        c.NQ = p.NQ;
        c.NQV = p.NQV;
        c.vrows = p.vrows;
        c.scale = scale;
        c.band = band;
        if ((e = launch_band_coef(c, p.NG, sms, status, st, coef_path)) != cudaSuccess) return e;
        // 2. the forward sweep, keeping what the adjoint needs
        const int64_t warps = (int64_t)sms * per_sm * BAND_WARPS;
        BandArgs f;
        memset(&f, 0, sizeof(f));
        f.src = src;
        f.band = band;
        f.n_pairs = m;
        f.ppw = (m + warps - 1) / warps;
        f.TperR = p.TperR;
        const int64_t nwarps = (m + f.ppw - 1) / f.ppw;
        const int64_t tm = f.ppw * p.TperR + 32;
        f.nck = (int)((tm + BAND_CK - 1) / BAND_CK);
        f.bq_stride = up4(tm * p.R + 1);
        if (nwarps * f.nck * 32 * 2 * p.R > rg.ckpt || nwarps * f.bq_stride > rg.botq)
            return cudaErrorInvalidValue;   // the workspace bound does not hold (cannot happen)
        f.ckpt = ckpt;
        f.exitk = exitk;
        f.botq = botq;
        f.out = out;   // the values too, when the caller asks (sigk_gram_value_and_grad)
        const int fgrid = (int)((nwarps + BAND_WARPS - 1) / BAND_WARPS);
        bool launched = false;
#define X(r, l, mb)                                                              \
        if (p.R == r && p.lam == l) {                                            \
            chain_band_kernel<r, l, mb, true><<<fgrid, BAND_WARPS * 32, 0, st>>>(f); \
            launched = true;                                                     \
        }
        SIGK_BAND_CASES(X)
#undef X
        if (!launched) return cudaErrorInvalidValue;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // 3. the adjoint sweep: dk/dc into gbar
        BandAdjArgs ad;
        ad.src = src;
        ad.band = band;
        ad.ckpt = ckpt;
        ad.exitk = exitk;
        ad.botq = botq;
        ad.nck = f.nck;
        ad.bq_stride = f.bq_stride;
        ad.gout = gout;
        ad.gband = gband;
        ad.n_pairs = m;
        ad.ppw = f.ppw;
        ad.TperR = p.TperR;
        ad.NQ = p.NQ;
        ad.NQV = p.NQV;
        ad.vrows = p.vrows;
        ad.nx = (int)nx;
        ad.ny = (int)ny;
        launched = false;
#define X(r, l, mb)                                                  \
        if (p.R == r && p.lam == l) {                                \
            if ((e = launch_adj<r, l>(ad, nwarps, st)) != cudaSuccess) return e; \
            launched = true;                                         \
        }
        SIGK_BAND_CASES(X)
#undef X
        if (!launched) return cudaErrorInvalidValue;
        if (rbf) {
            // the RBF lift: the chain rule through kappa over the points
            if ((e = rbf_chain_rule(src, p, m, a0, nA, nBall, kb, gband, gbar, dincA, dincB, rsum, part, dA, dB,
                                    add, sms, st)) != cudaSuccess)
                return e;
            continue;
        }
        // a Gram's contractions on the tensor cores (split-TF32) with the
        // tcgen05 path (coef_path 3), else on the FP32 pipe.  The tensor-core
        // contraction matches the FP32 one's accuracy but measured slower on
        // the 128 x 128 MMD Gram (2.6 against 1.5 ms a launch): its chunks run
        // in lockstep (copy, split, MMAs, read-back behind block barriers)
        const bool tc = bwd_dense_gbar(src0, coef_path);
        // 3b. dk/dc from the band layout into the dense Gbar (the tensor-core
        // contraction reads it; the FP32 one reads the band layout itself)
        if (tc) {
            // blocks below the diagonal of a symmetric Gram's dense dk/dc stay zero
            if (sym && cudaMemsetAsync(gbar, 0, sizeof(float) * rg.gbar, st) != cudaSuccess) return cudaErrorUnknown;
            BandGbarArgs gb;
            memset(&gb, 0, sizeof(gb));   // s_pair = 0: the dense Gbar, not the surface
            gb.src = src;
            gb.gband = gband;
            gb.gbar = gbar;
            gb.g_ld = gram ? nBall * ny : ny;
            gb.a_first = a0;
            gb.gram = gram ? 1 : 0;
            gb.n_pairs = m;
            gb.TperR = p.TperR;
            gb.NQV = p.NQV;
            gb.vrows = p.vrows;
            gb.nx = (int)nx;
            gb.ny = (int)ny;
            const int64_t tasks = m * gb_groups(p.TperR, false, p.NG);
            const int ggrid = (int)(tasks < (int64_t)sms * 8 ? tasks : (int64_t)sms * 8);
            if (p.NG == 8) band_gbar_kernel<8><<<ggrid, GB_THREADS, 0, st>>>(gb);
            else if (p.NG == 4) band_gbar_kernel<4><<<ggrid, GB_THREADS, 0, st>>>(gb);
            else band_gbar_kernel<2><<<ggrid, GB_THREADS, 0, st>>>(gb);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // 4. increments of this launch's paths
        band_inc_kernel<<<sms * 4, 256, 0, st>>>((const float *)src.A + a0 * src.La * d, nA, src.La, d, incA);
        if (!gram)
            band_inc_kernel<<<sms * 4, 256, 0, st>>>((const float *)src.B + src.kbase * src.Lb * d, m, src.Lb, d,
                                                     incB);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // 5. chain rule: dinc_A = gbar inc_B, dinc_B (+)= gbar^T inc_A
        GemmArgs g1;
        memset(&g1, 0, sizeof(g1));
        g1.G = gbar;
        g1.Bm = sym ? incA : incB;
        g1.C = dincA;
        g1.N = (int)d;
        g1.trans = 0;
        g1.tri_rb = sym ? nx : 0;
        g1.tri_cb = sym ? ny : 0;
        GemmArgs g2 = g1;
        g2.Bm = incA;
        g2.C = dincB;
        g2.trans = 1;
        int64_t batches;
        if (gram) {
            batches = 1;
            g1.g_ld = g2.g_ld = nBall * ny;
            g1.M = nA * nx; g1.K = nBall * ny;
            g2.M = nBall * ny; g2.K = nA * nx;
            g1.nA = g2.nA = nA;
            g1.nB = g2.nB = nBall;
        } else {
            batches = m;
            g1.b_bstride = ny * d; g2.b_bstride = nx * d;
            g1.c_bstride = nx * d; g2.c_bstride = ny * d;
            g1.M = nx; g1.K = ny;
            g2.M = ny; g2.K = nx;
            g1.nA = g2.nA = 1;
            g1.nB = g2.nB = 1;
        }
        // output tiles: 128 band coordinates of one output path (band rows,
        // or band columns when trans) by 32 channels
        const int64_t BHr = 32 * (int64_t)p.NG, NQc = (int64_t)p.TperR * p.NG;
        const int64_t tiles1 = (gram ? g1.nA : 1) * ((BHr + GT_M - 1) / GT_M);
        const int64_t tiles2 = (gram ? g2.nB : 1) * ((NQc + GT_M - 1) / GT_M);
        // a Gram's contractions have long reductions: split them to about four
        // blocks per SM, the partial tiles summed in a fixed order.  The Gram's
        // column-path gradients add up over launches.
        auto split = [&](int64_t tiles, int64_t nsl) {
            if (!gram) return 1;
            tiles *= (d + GT_N - 1) / GT_N;
            int64_t ksp = (4 * (int64_t)sms + tiles - 1) / tiles;
            if (ksp > nsl / 4) ksp = nsl / 4;
            if (ksp > GEMM_MAX_SPLIT) ksp = GEMM_MAX_SPLIT;
            return (int)(ksp < 1 ? 1 : ksp);
        };
        g1.ksplit = split(tiles1, nBall * ((NQc + GT_K - 1) / GT_K));
        g2.ksplit = split(tiles2, nA * (BHr / GT_K));
        g1.partial = g2.partial = part;
        const bool add_b = (gram && kb > 0) || sym;
        if (sym) g2.C = dincA;   // column-role gradients of the same paths: add them to the row role's
        // the split sum writes the result; an unsplit contraction that must add goes through it too
        if (add_b && g2.ksplit == 1) g2.ksplit = 2;
        const dim3 gd1((unsigned)tiles1, (unsigned)((d + GT_N - 1) / GT_N), (unsigned)(batches * g1.ksplit));
        const dim3 gd2((unsigned)tiles2, (unsigned)((d + GT_N - 1) / GT_N), (unsigned)(batches * g2.ksplit));
        // the FP32 contractions gather dk/dc from the band layout
        g1.band = g2.band = gband;
        g1.mode = g2.mode = src.mode;
        g1.nb = g2.nb = src0.nb;
        g1.a0 = g2.a0 = a0;
        g1.kbase = g2.kbase = src.kbase;
        g1.TperR1 = g2.TperR1 = p.TperR + 1;
        g1.vrows = g2.vrows = p.vrows;
        g1.NQV = g2.NQV = p.NQV;
        g1.nx = g2.nx = (int)nx;
        g1.ny = g2.ny = (int)ny;
        auto gemm = [&](const dim3 &gd, const GemmArgs &ga) {
            if (p.NG == 8) band_gemm_kernel<8><<<gd, 256, 0, st>>>(ga);
            else if (p.NG == 4) band_gemm_kernel<4><<<gd, 256, 0, st>>>(ga);
            else band_gemm_kernel<2><<<gd, 256, 0, st>>>(ga);
        };
        auto as_chain = [&](const GemmArgs &ga, int add) {
            ChainGemm cg;
            cg.G = ga.G;
            cg.g_ld = ga.g_ld;
            cg.trans = ga.trans;
            cg.Bm = ga.Bm;
            cg.C = ga.C;
            cg.M = ga.M;
            cg.K = ga.K;
            cg.N = ga.N;
            cg.add = add;
            cg.tri_rb = ga.tri_rb;
            cg.tri_cb = ga.tri_cb;
            return cg;
        };
        if (dA) {
            if (tc) {
                if ((e = launch_chain_gemm_tc5(as_chain(g1, 0), status, st)) != cudaSuccess) return e;
            } else {
                gemm(gd1, g1);
                if (g1.ksplit > 1)
                    band_split_sum_kernel<<<sms * 4, 256, 0, st>>>(part, g1.ksplit, g1.M * d, 0, dincA);
            }
        }
        if (dB || sym) {
            if (tc) {
                if ((e = launch_chain_gemm_tc5(as_chain(g2, add_b ? 1 : 0), status, st)) != cudaSuccess) return e;
            } else {
                gemm(gd2, g2);
                if (g2.ksplit > 1)
                    band_split_sum_kernel<<<sms * 4, 256, 0, st>>>(part, g2.ksplit, g2.M * d, add_b ? 1 : 0,
                                                                   g2.C);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // 6. point gradients
        if (dA)
            band_points_kernel<<<sms * 4, 256, 0, st>>>(dincA, nA, src.La, d, scale, add, dA + a0 * src.La * d);
        if (dB && !gram)
            band_points_kernel<<<sms * 4, 256, 0, st>>>(dincB, m, src.Lb, d, scale, add,
                                                      dB + src.kbase * src.Lb * d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (dB && gram && !rbf) {
        band_points_kernel<<<sms * 4, 256, 0, st>>>(dincB, nBall, src0.Lb, d, scale, add, dB);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}


}  // namespace sigk
