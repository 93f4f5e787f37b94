// Coarse-cell coefficients of the RBF-lifted scheme (Sec. 2.2): for every
// real coarse cell (p, q) of every pair, c = 1/2 4^-lambda x the second
// difference of kappa(a,b) = exp(-|a-b|^2 / (2 sigma^2)) over the cell's four
// corner points (rbf_second_difference), passed through the scheme's map
// (scheme_coef), and stored where the sweep that follows reads it.
//
// The kernel works on 32 x 32 tiles of a pair's coarse grid.  A block stages
// the tile's 33 row points and 33 column points in shared memory, 32 channels
// at a time, channel-major; thread t owns row t/8 and columns 4 (t%8) .. +3 of
// the tile and sums, per channel, the six inner products the second
// difference needs (|u|^2, <u,dx>, <u,dy>, <dx,dy> per cell, |dx|^2 per row,
// |dy|^2 per column, u = x_p - y_q): 1 subtraction and 4 FMAs per cell and
// channel.  Work units are (pair, tile) with the tile count of the largest
// pair; a unit past its pair's grid does nothing.
//
// The destination layout is a template parameter with two device calls:
//   Geo geo(int64_t k)                        pair k's row and column points
//                                             (rows, cols), coarse sizes (nx,
//                                             ny) and whatever store() needs
//   void store(const Geo &, int p, int q, T c) writes coarse cell (p, q)
// Entries that are not real cells (padding, virtual rows and columns) are not
// written: the caller zero-fills the destination first.
#pragma once
#include "sigk_internal.cuh"

namespace sigk {

constexpr int RBF_T = 32;     // tile side (coarse cells)
constexpr int RBF_CH = 32;    // channels staged per pass
constexpr int RBF_THREADS = 256;

template <typename T, class Layout>
__global__ void __launch_bounds__(RBF_THREADS) rbf_coef_kernel(Layout lay, int64_t n_pairs, int64_t tiles_r,
                                                               int64_t tiles_c, int64_t d, T s, T scale,
                                                               int scheme) {
    __shared__ T xs[RBF_CH][RBF_T + 1];
    __shared__ T ys[RBF_CH][RBF_T + 2];
    const int tid = threadIdx.x;
    const int r = tid >> 3, c0 = (tid & 7) * 4;
    const int64_t per_pair = tiles_r * tiles_c;
    const int64_t units = n_pairs * per_pair;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t k = u / per_pair;
        const int64_t t = u - k * per_pair;
        const typename Layout::Geo g = lay.geo(k);
        const int p0 = (int)(t / tiles_c) * RBF_T, q0 = (int)(t % tiles_c) * RBF_T;
        if (p0 >= g.nx || q0 >= g.ny) continue;   // block-uniform
        T uu[4], ux[4], uy[4], xy[4], ny[4], nx = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) { uu[j] = 0; ux[j] = 0; uy[j] = 0; xy[j] = 0; ny[j] = 0; }
        for (int64_t cb = 0; cb < d; cb += RBF_CH) {
            __syncthreads();
            // points p0 .. p0+32 and q0 .. q0+32 (0 past the path's last point)
            for (int v = tid; v < RBF_CH * (RBF_T + 1); v += RBF_THREADS) {
                const int i = v / RBF_CH, c = v - (v / RBF_CH) * RBF_CH;
                const bool cin = cb + c < d;
                xs[c][i] = (cin && p0 + i <= g.nx) ? g.rows[(int64_t)(p0 + i) * d + cb + c] : (T)0;
                ys[c][i] = (cin && q0 + i <= g.ny) ? g.cols[(int64_t)(q0 + i) * d + cb + c] : (T)0;
            }
            __syncthreads();
            const int nc = d - cb < RBF_CH ? (int)(d - cb) : RBF_CH;
            for (int c = 0; c < nc; ++c) {
                const T xa = xs[c][r], dxv = xs[c][r + 1] - xa;
                nx += dxv * dxv;
                T ya = ys[c][c0];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const T yb = ys[c][c0 + j + 1];
                    const T dyv = yb - ya, uv = xa - ya;
                    ny[j] += dyv * dyv;
                    uu[j] += uv * uv;
                    ux[j] += uv * dxv;
                    uy[j] += uv * dyv;
                    xy[j] += dxv * dyv;
                    ya = yb;
                }
            }
        }
        const int p = p0 + r;
        if (p < g.nx) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = q0 + c0 + j;
                if (q < g.ny) {
                    const T G = rbf_second_difference(uu[j], ux[j], uy[j], xy[j], nx, ny[j], s);
                    lay.store(g, p, q, scheme_coef(G * scale, scheme));
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
    const int64_t tr = (max_nx + RBF_T - 1) / RBF_T, tc = (max_ny + RBF_T - 1) / RBF_T;
    int64_t grid = n_pairs * tr * tc;
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    rbf_coef_kernel<T, Layout><<<(int)grid, RBF_THREADS, 0, st>>>(
        lay, n_pairs, tr, tc, d, (T)(0.5 / (sigma * sigma)), (T)scale, scheme);
    return cudaGetLastError();
}

}  // namespace sigk
