// placeholder until the tensor-core contraction lands
#include "common.cuh"
int wl_rows_split(cov_handle* h, cudaStream_t) { return wl_fail(h, COV_ERR_INVALID, "COV_SPLIT_BF16 not built"); }
int wl_syrk_tc(cov_handle* h, double*, int64_t, cudaStream_t) { return wl_fail(h, COV_ERR_INVALID, "COV_SPLIT_BF16 not built"); }
