// Internal declarations shared by the libils.so translation units.
#pragma once
#include <cuda_runtime.h>

#include "ils_fft.cuh"

namespace ils {

// Parameters of Eq. 7 for one image.
struct MuParams {
  float c;       // c0 = p eps^(p/2-1)  (Eq. 11)
  float p;
  float eps;
  float a;       // p/2 - 1
  float half_lambda;
};

// Launch geometry picked by the host planner (validated before any launch).
struct Geometry {
  int rows_fwd;      // output rows per CTA in the fused row pass (reads rows_fwd + 2 rows)
  int threads_row, ept_row;
  int rows_inv;      // rows per CTA in the final inverse row pass
  int threads_inv, ept_inv;
  int cols;          // complex columns per CTA in the column pass
  int threads_col, ept_col;
  size_t smem_fwd, smem_inv, smem_col;  // dynamic shared memory bytes
  int warp_row;      // index of a warp-per-row kernel for M = W/2, or -1
  int fixed_row;     // index of a compile-time row plan for M = W/2, or -1 (generic kernels)
  int fixed_col;     // index of a compile-time column plan for H, or -1
};

// Device tables for one (H, W, lambda, c).
struct Tables {
  float2* twW;   // W entries: exp(-2 pi i t / W)
  float2* twH;   // H entries: exp(-2 pi i t / H)
  float* ax;     // M+1 entries: lambda c (1 - cos(2 pi k / W)),  k = 0..M
  float* by;     // H entries:   lambda c (1 - cos(2 pi l / H)),  l = 0..H-1
};

struct ImageDesc {
  int H, W, C;
  FftPlan planM;  // length W/2 (row FFT on packed complex rows)
  FftPlan planH;  // length H   (column FFT)
};

bool make_fft_plan(int n, FftPlan* out);
bool pick_geometry(int H, int W, Geometry* g);

// Launchers (asynchronous on `stream`); return the launch error.
cudaError_t launch_row_forward(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float* f, const float* u0, const float2* spec_in, float2* spec_out,
                               float* u_ckpt, cudaStream_t stream);
cudaError_t launch_col_solve(const ImageDesc& d, const Geometry& g, const Tables& t, float2* spec,
                             cudaStream_t stream);
cudaError_t launch_row_inverse(const ImageDesc& d, const Geometry& g, const Tables& t, const float2* spec,
                               float* u, cudaStream_t stream);
cudaError_t launch_row_adjoint(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float2* spec_in, const float* u_n, float* fbar, bool fbar_first, float* gu0,
                               bool last, float2* spec_out, cudaStream_t stream);
cudaError_t set_kernel_attributes();
void record_cuda_error(const char* where, cudaError_t e);  // text for ils_last_error()
// 32->32 channel conv3x3 on tcgen05 tensor cores (ils_cnn_tc.cu)
bool conv32_tc_available();
cudaError_t conv32_tc_set_attributes();
cudaError_t launch_conv32_tc(int B, int H, int W, const void* in, const void* wt, const float* bias, void* out,
                             const void* mask, int relu, int* error, cudaStream_t st);
// max |a - b| over n floats as the bit pattern of a non-negative float, atomically max'ed into *out
cudaError_t launch_maxabsdiff(const float* a, const float* b, size_t n, unsigned int* out, cudaStream_t st);

// Compile-time specialised kernels (ils_kernels_fixed.cu).
int fixed_row_index(int M);
int fixed_col_index(int H);
int fixed_row_variants(int M, int* idx, int max);  // all entries for a length (first = default)
int fixed_col_variants(int H, int* idx, int max);
cudaError_t fixed_set_attributes();
cudaError_t fixed_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                              const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                              cudaStream_t stream);
cudaError_t fixed_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                              cudaStream_t stream);
cudaError_t fixed_col_solve(int idx, const ImageDesc& d, const Tables& t, float2* spec, cudaStream_t stream);

// Warp-per-row kernels (ils_rows_warp.cu).
int warp_row_variants(int M, int* idx, int max);
cudaError_t warp_set_attributes();
cudaError_t warp_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                             const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                             cudaStream_t stream);
cudaError_t warp_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                             cudaStream_t stream);

}  // namespace ils
