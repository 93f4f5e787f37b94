// Coarse-cell coefficients of the RBF-lifted scheme (Sec. 2.2): for every
// real coarse cell (p, q) of every pair, c = 1/2 4^-lambda x the second
// difference of kappa(a,b) = exp(-|a-b|^2 / (2 sigma^2)) over the cell's four
// corner points (rbf_second_difference), passed through the scheme's map
// (scheme_coef), and stored where the sweep that follows reads it.
//
// The kernel works on 32 NR x 32 tiles of a pair's coarse grid (NR = 4 rows
// per thread in f32, 2 in f64).  A block stages the tile's 32 NR + 1 row points
// and 33 column points in shared memory, 32 channels at a time,
// channel-major; thread t owns rows NR (t/8) .. +NR-1 and columns
// 4 (t%8) .. +3 of the tile and sums, per channel, the six inner
// products the second difference needs (|u|^2, <u,dx>, <u,dy>, <dx,dy> per
// cell, |dx|^2 per row, |dy|^2 per column, u = x_p - y_q): 1 subtraction and
// 4 FMAs per cell and channel.  Work units are (pair, tile) with the tile
// count of the largest pair; a unit past its pair's grid does nothing.
//
// The destination layout is a template parameter with three device calls:
//   Geo geo(int64_t k)               pair k's row and column points (rows,
//                                    cols), coarse sizes (nx, ny) and whatever
//                                    the stores need
//   Row row(const Geo &, int p)      what the stores of coarse row p share
//   void store(const Geo &, const Row &, int q, T c)   writes cell (p, q)
// Entries that are not real cells (padding, virtual rows and columns) are not
// written: the caller zero-fills the destination first.
#pragma once
#include "sigk_internal.cuh"

namespace sigk {

// rows per thread: 4 in f32, 2 in f64 (register budget); tile rows 32 x that
template <typename T>
__host__ __device__ constexpr int rbf_rows() { return sizeof(T) == 4 ? 4 : 2; }
constexpr int RBF_TC = 32;    // tile columns: 4 per thread
constexpr int RBF_CH = 32;    // channels staged per pass
constexpr int RBF_THREADS = 256;

template <typename T, class Layout>
__global__ void __launch_bounds__(RBF_THREADS) rbf_coef_kernel(Layout lay, int64_t n_pairs, int tiles_r,
                                                               int tiles_c, int64_t d, T s, T scale,
                                                               int scheme) {
    constexpr int NR = rbf_rows<T>(), TR = 32 * NR;
    __shared__ T xs[RBF_CH][TR + 1];
    __shared__ T ys[RBF_CH][RBF_TC + 2];
    const int tid = threadIdx.x;
    const int r = (tid >> 3) * NR, c0 = (tid & 7) * 4;
    const int per_pair = tiles_r * tiles_c;
    const int64_t units = n_pairs * per_pair;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        int64_t k;
        int t;
        if (units < (1LL << 31)) {   // 32-bit decode (the common case)
            k = (int)u / per_pair;
            t = (int)u - (int)k * per_pair;
        } else {
            k = u / per_pair;
            t = (int)(u - k * per_pair);
        }
        const typename Layout::Geo g = lay.geo(k);
        const int p0 = (t / tiles_c) * TR, q0 = (t - (t / tiles_c) * tiles_c) * RBF_TC;
        if (p0 >= g.nx || q0 >= g.ny) continue;   // block-uniform
        // points p0 .. p0 + TR and q0 .. q0 + 32 (0 past the path's last
        // point), channels cb .. cb + nc - 1: consecutive threads read
        // consecutive channels of a point
        auto stage = [&](int64_t cb, int nc) {
            __syncthreads();
            for (int v = tid; v < nc * (TR + 1); v += RBF_THREADS) {
                const int i = v / nc, c = v - i * nc;
                xs[c][i] = p0 + i <= g.nx ? g.rows[(int64_t)(p0 + i) * d + cb + c] : (T)0;
            }
            for (int v = tid; v < nc * (RBF_TC + 1); v += RBF_THREADS) {
                const int i = v / nc, c = v - i * nc;
                ys[c][i] = q0 + i <= g.ny ? g.cols[(int64_t)(q0 + i) * d + cb + c] : (T)0;
            }
            __syncthreads();
        };
        if constexpr (sizeof(T) == 4) {
            // f32: columns (j, j + 1) of a row share a float2, each sum a packed
            // FMA (the same operations per cell as the scalar loop below)
            float2 uu2[NR][2], ux2[NR][2], uy2[NR][2], xy2[NR][2], ny2[2];
            float nxs[NR];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                ny2[h] = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    uu2[i][h] = ny2[h]; ux2[i][h] = ny2[h]; uy2[i][h] = ny2[h]; xy2[i][h] = ny2[h];
                }
            }
#pragma unroll
            for (int i = 0; i < NR; ++i) nxs[i] = 0.f;
            for (int64_t cb = 0; cb < d; cb += RBF_CH) {
                const int nc = d - cb < RBF_CH ? (int)(d - cb) : RBF_CH;
                stage(cb, nc);
#pragma unroll 2
                for (int c = 0; c < nc; ++c) {
                    float xv[NR + 1], yv[5];
#pragma unroll
                    for (int i = 0; i <= NR; ++i) xv[i] = xs[c][r + i];
#pragma unroll
                    for (int j = 0; j < 5; ++j) yv[j] = ys[c][c0 + j];
                    float2 ny_[2], dy2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        ny_[h] = make_float2(-yv[2 * h], -yv[2 * h + 1]);
                        dy2[h] = make_float2(yv[2 * h + 1] - yv[2 * h], yv[2 * h + 2] - yv[2 * h + 1]);
                        ny2[h] = __ffma2_rn(dy2[h], dy2[h], ny2[h]);
                    }
#pragma unroll
                    for (int i = 0; i < NR; ++i) {
                        const float dxv = xv[i + 1] - xv[i];
                        nxs[i] = fmaf(dxv, dxv, nxs[i]);
                        const float2 x2 = make_float2(xv[i], xv[i]), d2 = make_float2(dxv, dxv);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 uv = __fadd2_rn(x2, ny_[h]);
                            uu2[i][h] = __ffma2_rn(uv, uv, uu2[i][h]);
                            ux2[i][h] = __ffma2_rn(uv, d2, ux2[i][h]);
                            uy2[i][h] = __ffma2_rn(uv, dy2[h], uy2[i][h]);
                            xy2[i][h] = __ffma2_rn(d2, dy2[h], xy2[i][h]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int p = p0 + r + i;
                if (p >= g.nx) break;
                const typename Layout::Row row = lay.row(g, p);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = q0 + c0 + j;
                    if (q < g.ny) {
                        const int h = j >> 1;
                        const bool hi = j & 1;
                        const float G = rbf_second_difference(
                            hi ? uu2[i][h].y : uu2[i][h].x, hi ? ux2[i][h].y : ux2[i][h].x,
                            hi ? uy2[i][h].y : uy2[i][h].x, hi ? xy2[i][h].y : xy2[i][h].x, nxs[i],
                            hi ? ny2[h].y : ny2[h].x, (float)s);
                        lay.store(g, row, q, scheme_coef(G * (float)scale, scheme));
                    }
                }
            }
            continue;
        }
        T uu[NR][4], ux[NR][4], uy[NR][4], xy[NR][4], ny[4], nx[NR];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ny[j] = 0;
#pragma unroll
            for (int i = 0; i < NR; ++i) { uu[i][j] = 0; ux[i][j] = 0; uy[i][j] = 0; xy[i][j] = 0; }
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) nx[i] = 0;
        for (int64_t cb = 0; cb < d; cb += RBF_CH) {
            const int nc = d - cb < RBF_CH ? (int)(d - cb) : RBF_CH;
            stage(cb, nc);
#pragma unroll 2
            for (int c = 0; c < nc; ++c) {
                T xv[NR + 1], dxv[NR];
#pragma unroll
                for (int i = 0; i <= NR; ++i) xv[i] = xs[c][r + i];
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    dxv[i] = xv[i + 1] - xv[i];
                    nx[i] += dxv[i] * dxv[i];
                }
                T ya = ys[c][c0];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const T yb = ys[c][c0 + j + 1];
                    const T dyv = yb - ya;
                    ny[j] += dyv * dyv;
#pragma unroll
                    for (int i = 0; i < NR; ++i) {
                        const T uv = xv[i] - ya;
                        uu[i][j] += uv * uv;
                        ux[i][j] += uv * dxv[i];
                        uy[i][j] += uv * dyv;
                        xy[i][j] += dxv[i] * dyv;
                    }
                    ya = yb;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int p = p0 + r + i;
            if (p >= g.nx) break;
            const typename Layout::Row row = lay.row(g, p);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = q0 + c0 + j;
                if (q < g.ny) {
                    const T G = rbf_second_difference(uu[i][j], ux[i][j], uy[i][j], xy[i][j], nx[i], ny[j], s);
                    lay.store(g, row, q, scheme_coef(G * scale, scheme));
                }
            }
        }
    }
}

// Zero-fill `zero_bytes` at `dst_zero`, then the coefficients of n_pairs
// pairs whose coarse grids are at most max_nx x max_ny.
template <typename T, class Layout>
cudaError_t launch_rbf_coef(const Layout &lay, int64_t n_pairs, int64_t max_nx, int64_t max_ny, int64_t d,
                            double sigma, double scale, int scheme, void *dst_zero, size_t zero_bytes,
                            int sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(dst_zero, 0, zero_bytes, st);
    if (e != cudaSuccess) return e;
    if (n_pairs <= 0 || max_nx <= 0 || max_ny <= 0) return cudaSuccess;
    constexpr int TR = 32 * rbf_rows<T>();
    const int64_t tr = (max_nx + TR - 1) / TR, tc = (max_ny + RBF_TC - 1) / RBF_TC;
    int64_t grid = n_pairs * tr * tc;
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    rbf_coef_kernel<T, Layout><<<(int)grid, RBF_THREADS, 0, st>>>(
        lay, n_pairs, (int)tr, (int)tc, d, (T)(0.5 / (sigma * sigma)), (T)scale, scheme);
    return cudaGetLastError();
}

}  // namespace sigk
