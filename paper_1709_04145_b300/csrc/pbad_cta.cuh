// Dense algebra of the Newton (LM) solve by a whole CTA: the Gram matrix
// J^T J as a tiled syrk and the Cholesky factorisation and solves of the
// damped system (Section 5, LM). Used by the CTA-mode Newton rollout and by
// pbad_damped_gram_solve.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pbad {

// Dense algebra of one instance by a whole CTA (all threads call; every
// branch is CTA-uniform). Jc: Jr column-major (column c at Jc + c Sn), H
// row-major, A the Cholesky factor stored column-major (L[r][c] at A[c Sn + r]).
namespace cta {
constexpr int kTile = 64, kChunk = 16, kPad = kChunk + 1;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += red[k];  // same order on every thread
  return t;
}
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
  for (int k = 1; k < nw; ++k) t = fmax(t, red[k]);
  return t;
}

// H = Jc^T Jc as a syrk: H[a][c] = sum_r Jc[a Sn + r] Jc[c Sn + r], on
// kTile x kTile tiles of the lower triangle (mirrored), the k dimension in
// chunks staged through shared memory (coalesced rows of Jc); each thread
// accumulates a 4 x 8 block in registers. blockDim.x must be 128.
__device__ inline void syrk(const double* Jc, double* H, int Sn, double* sa, double* sc) {
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;  // 16 x 8 threads, 4 x 8 outputs each
  const int nt = (Sn + kTile - 1) / kTile;
  for (int ta = 0; ta < nt; ++ta)
    for (int tc = 0; tc <= ta; ++tc) {
      const int a0 = ta * kTile, c0 = tc * kTile;
      double acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
      for (int k0 = 0; k0 < Sn; k0 += kChunk) {
        __syncthreads();
        for (int e = tid; e < kTile * kChunk; e += blockDim.x) {
          const int row = e / kChunk, k = e - row * kChunk;
          const int ra = a0 + row, rc = c0 + row, kk = k0 + k;
          sa[row * kPad + k] = (ra < Sn && kk < Sn) ? Jc[(int64_t)ra * Sn + kk] : 0.0;
          sc[row * kPad + k] = (rc < Sn && kk < Sn) ? Jc[(int64_t)rc * Sn + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kChunk; ++k) {
          double av[4], cv[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = sa[(ty * 4 + i) * kPad + k];
#pragma unroll
          for (int j = 0; j < 8; ++j) cv[j] = sc[(tx * 8 + j) * kPad + k];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int a = a0 + ty * 4 + i, c = c0 + tx * 8 + j;
          if (a < Sn && c < Sn && c <= a) {
            H[(int64_t)a * Sn + c] = acc[i][j];
            H[(int64_t)c * Sn + a] = acc[i][j];
          }
        }
    }
  __syncthreads();
}

// Cholesky of H + lambda I, blocked left-looking by panels of kTile
// columns: each panel is first updated by the columns to its left as
// kTile x kTile tiles staged through shared memory (sa, sc; each thread a
// 4 x 8 register block, the rows of one column of the column-major factor
// read contiguously), then factored column by column within itself. Then
// dl = -(H + lambda I)^-1 gg by forward and back substitution. Returns false
// (on every thread) if a pivot is not positive. vec: Sn doubles of shared
// memory, red: reduction scratch. blockDim.x must be 128.
__device__ inline bool factor_solve(const double* H, double* A, const double* gg, double* dl, int Sn,
                             double lambda, double* vec, double* red, double* sa, double* sc) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ty = tid >> 3, tx = tid & 7;
  __shared__ double s_piv;
  for (int j0 = 0; j0 < Sn; j0 += kTile) {
    const int jw = min(kTile, Sn - j0);
    // the panel's columns of H + lambda I (rows from the diagonal down)
    for (int c = 0; c < jw; ++c) {
      const int j = j0 + c;
      for (int r = j + tid; r < Sn; r += nth)
        A[(int64_t)j * Sn + r] = H[(int64_t)j * Sn + r] + (r == j ? lambda : 0.0);
    }
    // minus L[r][0:j0] L[j0 + c][0:j0]^T for the rows r >= j0
    if (j0 > 0) {
      for (int r0 = j0; r0 < Sn; r0 += kTile) {
        double acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[i][q] = 0.0;
        for (int k0 = 0; k0 < j0; k0 += kChunk) {
          __syncthreads();
          for (int e = tid; e < kTile * kChunk; e += nth) {
            const int k = e / kTile, row = e - k * kTile;  // rows fastest: contiguous in A
            const int kk = k0 + k, ra = r0 + row, rc = j0 + row;
            sa[row * kPad + k] = (ra < Sn && kk < j0) ? A[(int64_t)kk * Sn + ra] : 0.0;
            sc[row * kPad + k] = (row < jw && kk < j0) ? A[(int64_t)kk * Sn + rc] : 0.0;
          }
          __syncthreads();
#pragma unroll 4
          for (int k = 0; k < kChunk; ++k) {
            double av[4], cv[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = sa[(ty * 4 + i) * kPad + k];
#pragma unroll
            for (int q = 0; q < 8; ++q) cv[q] = sc[(tx * 8 + q) * kPad + k];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int q = 0; q < 8; ++q) acc[i][q] = fma(av[i], cv[q], acc[i][q]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int r = r0 + ty * 4 + i, c = tx * 8 + q;
            if (r < Sn && c < jw && r >= j0 + c) A[(int64_t)(j0 + c) * Sn + r] -= acc[i][q];
          }
      }
      __syncthreads();
    }
    // the panel itself, one column per pass (row j of the panel's L in vec)
    for (int c = 0; c < jw; ++c) {
      const int j = j0 + c;
      for (int k = j0 + tid; k < j; k += nth) vec[k - j0] = A[(int64_t)k * Sn + j];
      __syncthreads();
      for (int r = j + tid; r < Sn; r += nth) {
        double t = A[(int64_t)j * Sn + r];
        for (int k = j0; k < j; ++k) t = fma(-A[(int64_t)k * Sn + r], vec[k - j0], t);
        if (r == j) s_piv = t;
        A[(int64_t)j * Sn + r] = t;
      }
      __syncthreads();
      const double d = s_piv;
      if (!(d > 0.0)) return false;  // CTA-uniform
      const double ljj = sqrt(d), inv = 1.0 / ljj;
      for (int r = j + 1 + tid; r < Sn; r += nth) A[(int64_t)j * Sn + r] *= inv;
      if (tid == 0) A[(int64_t)j * Sn + j] = ljj;
      __syncthreads();
    }
  }
  // L y = -gg, column by column
  for (int k = tid; k < Sn; k += nth) vec[k] = -gg[k];
  __syncthreads();
  for (int k = 0; k < Sn; ++k) {
    const double yk = vec[k] / A[(int64_t)k * Sn + k];
    __syncthreads();
    for (int r = k + 1 + tid; r < Sn; r += nth) vec[r] = fma(-A[(int64_t)k * Sn + r], yk, vec[r]);
    if (tid == 0) vec[k] = yk;
    __syncthreads();
  }
  // L^T x = y, row by row: x_r = (y_r - sum_{k > r} L[k][r] x_k) / L[r][r]
  for (int r = Sn - 1; r >= 0; --r) {
    double s = 0.0;
    for (int k = r + 1 + tid; k < Sn; k += nth) s = fma(A[(int64_t)r * Sn + k], vec[k], s);
    s = block_sum(s, red);
    const double xr = (vec[r] - s) / A[(int64_t)r * Sn + r];
    __syncthreads();
    if (tid == 0) vec[r] = xr;
    __syncthreads();
  }
  for (int k = tid; k < Sn; k += nth) dl[k] = vec[k];
  __syncthreads();
  return true;
}
}  // namespace cta

}  // namespace pbad
