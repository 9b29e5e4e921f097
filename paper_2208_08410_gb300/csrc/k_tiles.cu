// The Gram operator of the orthogonal batching (Sec. V-C, Fig. 2c-d, Alg. 3):
// the n x n Gram matrix is held as FP64 tiles B_JI = A_J^T A_I (J <= I, the
// symmetric task reuse) of a bs-column partition of A, and one application
// w = G v is
//     w_J += B_JI v_I   and, for J < I,   w_I += B_JI^T v_J
// over the stored tiles.  A diagonal tile holds its upper triangle (entries
// a <= b) and zeros below, so its transposed part takes only a < b.  Sums
// are FP64; each tile's row and column sums are added into w (FP64) with
// atomics.  The last kernel rounds w to the FP32 iterate the vector kernels
// take and forms v . w (FP64), which is v^T G v for the Rayleigh quotient.
#include "common.cuh"

namespace tsvd {
namespace {

constexpr int kTileRows = 32;   // rows of a tile per CTA
constexpr int kTileCols = 256;  // columns per CTA (one per thread)

__global__ void __launch_bounds__(kTileCols) tile_symv_kernel(const double *__restrict__ T, int64_t ldt, int nJ,
                                                              int nI, const float *__restrict__ vJ,
                                                              const float *__restrict__ vI, double *__restrict__ wJ,
                                                              double *__restrict__ wI, int diag) {
  __shared__ double rsum[kTileCols / 32][kTileRows];
  const int b = blockIdx.x * kTileCols + threadIdx.x;
  const int a0 = blockIdx.y * kTileRows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool colok = b < nI;
  const double vb = colok ? (double)vI[b] : 0.0;
  double csum = 0.0;
#pragma unroll 4
  for (int r = 0; r < kTileRows; ++r) {
    const int a = a0 + r;
    double x = 0.0;
    if (a < nJ && colok) x = T[(int64_t)a * ldt + b];
    // row part: B[a][b] v_I[b]
    double t = x * vb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) rsum[warp][r] = t;
    // column part: B[a][b] v_J[a] (strictly above the diagonal of a diagonal tile)
    if (a < nJ && (!diag || a < b)) csum = fma(x, (double)vJ[a], csum);
  }
  __syncthreads();
  if (threadIdx.x < kTileRows) {
    const int a = a0 + threadIdx.x;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kTileCols / 32; ++w) t += rsum[w][threadIdx.x];
    if (a < nJ && t != 0.0) atomicAdd(wJ + a, t);
  }
  if (colok && csum != 0.0) atomicAdd(wI + b, csum);
}

__global__ void tile_finish_kernel(int64_t n, const float *__restrict__ v, const double *__restrict__ w64,
                                   float *__restrict__ w, double *__restrict__ ss) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = w64[i];
    w[i] = (float)x;
    s = fma((double)v[i], x, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(ss, s);
}

}  // namespace

tsvd_status launch_tile_symv(const double *T, int64_t ldt, int64_t nJ, int64_t nI, const float *vJ, const float *vI,
                             double *wJ, double *wI, bool diag, cudaStream_t stream) {
  if (nJ <= 0 || nI <= 0) return TSVD_OK;
  if (nJ > 0x7fffffffLL || nI > 0x7fffffffLL) return TSVD_EUNSUPPORTED;
  const int64_t gy = ceil_div(nJ, kTileRows), gx = ceil_div(nI, kTileCols);
  if (gy > 65535) return TSVD_EUNSUPPORTED;
  tile_symv_kernel<<<dim3((unsigned)gx, (unsigned)gy), kTileCols, 0, stream>>>(T, ldt, (int)nJ, (int)nI, vJ, vI, wJ,
                                                                              wI, diag ? 1 : 0);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

tsvd_status launch_tile_finish(int64_t n, const float *v, const double *w64, float *w, double *ss,
                               cudaStream_t stream) {
  if (n <= 0) return TSVD_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), 1024);
  tile_finish_kernel<<<(unsigned)blocks, 256, 0, stream>>>(n, v, w64, w, ss);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
