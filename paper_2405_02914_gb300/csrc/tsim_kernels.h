// tsim_kernels.h -- host-side launchers of the sm_103a kernels (tsim_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "tsim_device.cuh"

namespace tsim {

enum { MODE_PROLOGUE_ = 0, MODE_ITER_ = 1, MODE_COMMIT_ = 2 };

void launch_round_begin(const Dev &d, cudaStream_t s);
void launch_set_end(const Dev &d, long long n, cudaStream_t s);
void grid_launch_shape(const Dev &d, long long max_nodes, int threads, int flat, dim3 &grid, dim3 &block);
void launch_grid(const Dev &d, long long max_nodes, int threads, int flat, cudaStream_t s);
void launch_transfer(const Dev &d, int mode, int block_offset, int nblocks, cudaStream_t s);
void launch_object_p2g(const Dev &d, int mode, int inst0, int rows, int max_obj, cudaStream_t s);
void *fn_object_p2g(int mode);
void launch_bin_staged(const Dev &d, int inst, int n, int par, cudaStream_t s);
void launch_gather(const Dev &d, int inst, long long positions, int par, cudaStream_t s);
void launch_pick(const Dev &d, int inst, const int *ids, int m, float *out, cudaStream_t s);
void launch_surface(const Dev &d, int inst, long long positions, int par, float *num, float *den, float *h,
                    float *nrm, int W, int H, float pitch, float h_empty, cudaStream_t s);

void launch_surface_disp(const Dev &d, int inst, long long positions, int par, const float *xref, float *acc,
                         float *u, int W, int H, float pitch, cudaStream_t s);
void launch_indenter_height(const Dev &d, int inst, float *h, int W, int H, float pitch, float clip, cudaStream_t s);
cudaError_t setup_kernels();
size_t transfer_smem_bytes();
int block_slots();

void *fn_round_begin();
void *fn_grid(int flat);
unsigned int round_begin_ctas(const Dev &d);
void *fn_transfer(int mode);
void *fn_spill(int mode);

}  // namespace tsim
