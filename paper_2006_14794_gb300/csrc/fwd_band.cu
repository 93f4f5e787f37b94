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

#include "sigk_internal.cuh"

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
            if (pos < a.TperR && pos > 0) {
                float4 *dst = reinterpret_cast<float4 *>(a.band + (((k * a.TperR + pos) * 32) + l) * SLOT);
                if constexpr (NG >= 4) {
#pragma unroll
                    for (int w = 0; w < NG; ++w)
#pragma unroll
                        for (int h = 0; h < NG / 4; ++h)
                            dst[w * (NG / 4) + h] = make_float4(acc[w][4 * h] * a.scale, acc[w][4 * h + 1] * a.scale,
                                                                acc[w][4 * h + 2] * a.scale, acc[w][4 * h + 3] * a.scale);
                } else {
                    dst[0] = make_float4(acc[0][0] * a.scale, acc[0][1] * a.scale, acc[1][0] * a.scale,
                                         acc[1][1] * a.scale);
                }
            } else if (pos == 0) {
                // the pair's own cells (w >= g); the cells w < g belong to the
                // previous pair's block, which writes them (pair 0: zeros)
                float *dst = a.band + ((k * a.TperR) * 32 + l) * SLOT;
#pragma unroll
                for (int w = 0; w < NG; ++w)
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (w >= g) dst[w * NG + g] = acc[w][g] * a.scale;
                        else if (k == 0) dst[w * NG + g] = 0.f;
                    }
            } else {
                // pos == TperR: the tail (w < g) into slot 0 of the next pair; after
                // the last pair the slot has no owner, so its own cells are zeroed
                float *dst = a.band + (((k + 1) * a.TperR) * 32 + l) * SLOT;
#pragma unroll
                for (int w = 0; w < NG; ++w)
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (w < g) dst[w * NG + g] = acc[w][g] * a.scale;
                        else if (k == a.n_pairs - 1) dst[w * NG + g] = 0.f;
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
};

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

// The sweep: fwd_chain.cu's chain_f32_kernel with its staging and dot
// products replaced by one coefficient vector per window, prefetched one
// macro-step ahead into the registers the window has just consumed.
template <int R, int LAM, int MINB>
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

    for (int64_t m = 0; m < total_m; ++m) {
        const bool trans = (pos == 0);
        const float *pn = (pos + 1 == TperR) ? slot(kl + 1, 0) : slot(kl, pos + 1);

#pragma unroll
        for (int w = 0; w < NG; ++w) {
#pragma unroll
            for (int g = 0; g < NH; ++g) {
                CO[g] = CN[g];
                CN[g] = make_float2(cb[w][g], cb[w][g + NH]);
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
                                const PairRef pr = pair_ref(a.src, k0 + kp);
                                a.out[pr.out0] = KP[i].y;
                                if (pr.out1 >= 0) a.out[pr.out1] = KP[i].y;
                            }
                        }
                    }
                }
                pK = (lane == 0) ? 1.f : shK;
                pQ = (lane == 0) ? 0.f : shQ;
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chain_band_kernel<R, LAM, MINB>,
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

int64_t band_bytes(const BandPlan &p, int64_t n_pairs) {
    return (int64_t)sizeof(float) * (n_pairs * p.TperR + 1) * p.slot_floats;
}

cudaError_t launch_band_f32(const PairSrc &src, const BandPlan &p, int64_t n_pairs, float *out,
                            void *ws, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    BandCoefArgs c;
    c.src = src;
    c.n_pairs = n_pairs;
    c.TperR = p.TperR;
    c.NQ = p.NQ;
    c.NQV = p.NQV;
    c.vrows = p.vrows;
    c.scale = 0.5f / (float)(1 << (2 * p.lam));
    c.band = (float *)ws;
    if (p.NG == 8) e = launch_coef<8>(c, sms, st);
    else if (p.NG == 4) e = launch_coef<4>(c, sms, st);
    else e = launch_coef<2>(c, sms, st);
    if (e != cudaSuccess) return e;

    const int per_sm = band_occupancy_of(p.R, p.lam);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t warps = (int64_t)sms * per_sm * BAND_WARPS;
    BandArgs a;
    a.src = src;
    a.out = out;
    a.band = (const float *)ws;
    a.n_pairs = n_pairs;
    a.ppw = (n_pairs + warps - 1) / warps;
    a.TperR = p.TperR;
    const int64_t nwarps = (n_pairs + a.ppw - 1) / a.ppw;
    const int grid = (int)((nwarps + BAND_WARPS - 1) / BAND_WARPS);
#define X(r, l, mb)                                                          \
    if (p.R == r && p.lam == l) {                                            \
        chain_band_kernel<r, l, mb><<<grid, BAND_WARPS * 32, 0, st>>>(a);    \
        return cudaGetLastError();                                           \
    }
    SIGK_BAND_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace sigk
