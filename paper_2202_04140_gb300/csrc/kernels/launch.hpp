// Host-callable launchers of the device kernels (internal to libace).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../../include/ace.h"

namespace ace {

namespace dev {
struct LoeArgs;
}

// Returns the fused kernel instantiation for (dtype, E, NOUT, grad, readout) or
// nullptr when that combination is not compiled; *nt receives its block size.
const void* fused_kernel_ptr(int dtype, int E, int nout, bool grad, int readout, int* nt);

// One-environment-per-lane variant (loe.cu): kernel, shared memory, entry binding.
const void* loe_kernel_ptr(bool grad, int readout, bool global, int* nt);
size_t loe_smem(int n_slots, int n_g, bool grad, int nt);
size_t loe_global_smem(int nt);
size_t loe_global_bytes_per_cta(int n_slots, int n_g, bool grad);
// Fill the per-warp task streams of the one-environment-per-lane kernel with the
// coefficients c (FP32, one channel): task t's header at item hpos[t], its entry
// pairs (entries toff[t] .. toff[t+1], an even count) in the items after it.
cudaError_t launch_bind_loe(const float* c, const int4* tasks, const int32_t* toff, const int32_t* col,
                            const int32_t* ebasis, const uint8_t* ew2, const int32_t* slot_basis,
                            const int32_t* hpos, int32_t n_tasks, int4* stream, cudaStream_t st);

// Two environments per lane, global workspace (loe_wide.cu): kernel, shared memory, workspace
// bytes per CTA (64 environments).
const void* loe_wide_kernel_ptr(bool grad, int readout, int* nt);
size_t loe_wide_smem(int nt);
size_t loe_wide_bytes_per_cta(int n_slots, int n_g, bool grad);

// Several channels, one environment per lane (loe_multi.cu, forward only): kernel, shared
// memory, launch with the index-bound streams and the coefficient table c[n_basis][16].
const void* loe_multi_kernel_ptr(int readout, int* nt);
size_t loe_multi_smem(int nt);
cudaError_t launch_loe_multi(const void* kernel, int grid, int nt, size_t smem, const dev::LoeArgs& base,
                             const int4* istream, const float* cvals, int n_out, cudaStream_t st);
// The per-warp streams bound with basis indices (bit 30: doubled) in place of coefficients.
cudaError_t launch_bind_loe_idx(const int4* tasks, const int32_t* toff, const int32_t* col, const int32_t* ebasis,
                                const uint8_t* ew2, const int32_t* slot_basis, const int32_t* hpos, int32_t n_tasks,
                                int4* stream, cudaStream_t st);

// Write the items of the per-warp streams that the binding does not touch (block headers and
// their columns): stream[pos[i]] = val[i].
cudaError_t launch_loe_static(const int32_t* pos, const int4* val, int32_t n, int4* stream, cudaStream_t st);

cudaError_t launch_bind(int dtype, const void* c, int n_out, int nout_pad, const int32_t* ebasis, const uint8_t* ew2,
                        int64_t n_entries, void* vals, const int32_t* lin_basis, int64_t n_lin, void* lin,
                        cudaStream_t st);

cudaError_t launch_plain_f64(const double* A, const double* c, const double* phibar, int64_t n_env, int n_out, int K,
                             int64_t n_nodes, const int32_t* left, const int32_t* right, const int32_t* node_basis,
                             double* phi, double* dA, double* AA, double* abar, cudaStream_t st);

// Fixed device scratch of ace_eval_plain_f64_static (plain_static.cu).
size_t static_scratch_bytes();
cudaError_t static_scratch_ptr(void** out);

cudaError_t launch_fma_probe(int64_t iters, int blocks, int threads, float* out, cudaStream_t st);

cudaError_t launch_pool(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, float rc, int nmin,
                        int nmax, int lmax, int kmax, float* A, cudaStream_t st);

// Fused forces pipeline (pool.cu): shared memory per CTA for this graph and these pooling
// parameters (0: the request does not fit the fused kernel), and its launch (one tile of 32
// environments per CTA iteration; b carries the graph, phi and the tile count).
size_t forces_fused_smem(int n_slots, int n_g, int K, int nmin, int nmax, int lmax, int kmax);
cudaError_t launch_forces_fused(const dev::LoeArgs& b, const float* pos, const int64_t* offsets, float rc, int nmin,
                                int nmax, int lmax, int readout, float* forces, int grid, size_t smem,
                                cudaStream_t st);
cudaError_t launch_pool_grad(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, float rc,
                             int nmin, int nmax, int lmax, int kmax, const float* dA, float alpha, float* dpos,
                             cudaStream_t st);

}  // namespace ace
