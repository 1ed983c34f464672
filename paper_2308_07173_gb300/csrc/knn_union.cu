// Search kernels over a map grown by appended points (pc_target_append):
// the main grid and the appended-points grid searched as one map in the
// same lane and warp paths as the whole-map kernels (knn_kernels.cuh,
// DEL = true).  This unit holds the whole-map variant; knn_union_win.cu the
// window variant.  Both compile in parallel with the other search units.
#include "knn_kernels.cuh"

void* pc_knn_union_kernel(int mode, bool with_cov) { return knn_union_kernel<false>(mode, with_cov); }

cudaError_t pc_knn_union_attrs() { return allow_union_smem<false>(); }
