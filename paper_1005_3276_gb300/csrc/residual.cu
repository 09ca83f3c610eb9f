// FP64 true residuals ||b - (M^dag M + shift) x|| / ||b|| of device fields.
#include "apply_impl.cuh"
#include "solver.h"
#include "wz_cg.cuh"

namespace wz {

// Per-system |b - (Ax + sigma x)|^2 and |b|^2 (FP64), one block per system;
// Ax = M^dag M x.
__global__ void residual_norms_kernel(const cplx<double>* b, const cplx<double>* Ax, const cplx<double>* x,
                                      long n_per_rhs, ShiftSpec sh, double* out) {
  __shared__ double red[33];
  const long off = (long)blockIdx.x * n_per_rhs;
  const long boff = sh.src(blockIdx.x) * n_per_rhs;
  const double sigma = sh.of(blockIdx.x);
  double rr = 0.0, bb = 0.0;
  for (long i = threadIdx.x; i < n_per_rhs; i += blockDim.x) {
    const cplx<double> bv = b[boff + i], av = Ax[off + i], xv = x[off + i];
    const double dx = bv.x - av.x - sigma * xv.x, dy = bv.y - av.y - sigma * xv.y;
    rr += dx * dx + dy * dy;
    bb += bv.x * bv.x + bv.y * bv.y;
  }
  rr = block_sum(rr, red);
  __syncthreads();
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = rr;
    out[2 * blockIdx.x + 1] = bb;
  }
}

// FP64 true relative residuals of (M^dag M + sigma_q) x_q = b_q (device fields).
int true_residuals(wz_ctx* c, const cplx<double>* b, const cplx<double>* x, int nrhs, const ShiftSpec& sh,
                   double* rel_out) {
  const size_t field = sizeof(cplx<double>) * 4 * (size_t)c->V * nrhs;
  WZ_CUDA_TRY(c, c->ws_apply.reserve(apply_ws_bytes<double>(c, WZ_OP_MDAGM, nrhs) + field));
  cplx<double>* Ax = (cplx<double>*)((char*)c->ws_apply.ptr + apply_ws_bytes<double>(c, WZ_OP_MDAGM, nrhs));
  int rc = apply_op<double>(c, WZ_OP_MDAGM, x, Ax, nrhs, 0.0, (cplx<double>*)c->ws_apply.ptr);
  if (rc) return rc;
  if (sizeof(double) * 2 * nrhs > WZ_PINNED_BYTES - WZ_PINNED_SCRATCH_OFFSET)
    return set_error(c, WZ_EINVAL, "too many right-hand sides");
  WZ_CUDA_TRY(c, c->ws_red.reserve(sizeof(double) * 2 * nrhs));
  count_launch();
  residual_norms_kernel<<<nrhs, 256, 0, c->stream>>>(b, Ax, x, 4L * c->V, sh, (double*)c->ws_red.ptr);
  WZ_CUDA_TRY(c, cudaGetLastError());
  double* h = (double*)((char*)c->host_pinned + WZ_PINNED_SCRATCH_OFFSET);  // not the solver-state region
  WZ_CUDA_TRY(c, cudaMemcpyAsync(h, c->ws_red.ptr, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, c->stream));
  WZ_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int j = 0; j < nrhs; ++j) rel_out[j] = h[2 * j + 1] > 0 ? sqrt(h[2 * j] / h[2 * j + 1]) : 0.0;
  return WZ_OK;
}

}  // namespace wz
