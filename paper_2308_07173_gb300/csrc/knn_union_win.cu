// Window variant of the union search kernels (knn_union.cu): rows on the
// window's boundary cells of either grid test each point against the window.
#include "knn_kernels.cuh"

void* pc_knn_union_kernel_win(int mode, bool with_cov) { return knn_union_kernel<true>(mode, with_cov); }

cudaError_t pc_knn_union_win_attrs() { return allow_union_smem<true>(); }
