// Window variant of the search kernels (pc_set_window): the same code as
// the whole-map kernels with WIN = true, so rows on the window's boundary
// cells test each point against the window box.
#include "knn_kernels.cuh"

void* pc_knn_kernel_win(int mode, bool with_cov, bool batch, bool stage) {
    return knn_kernel<true>(mode, with_cov, batch, stage);
}

cudaError_t pc_knn_win_attrs() { return allow_all_smem<true>(); }
