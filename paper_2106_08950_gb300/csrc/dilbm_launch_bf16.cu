// Step-sweep and batched-sweep launchers for __nv_bfloat16 storage, every launch
// shape (warps per block 2, 4, 8; with and without edge handling).  One
// translation unit per storage type so that the library compiles in parallel.
#include "dilbm_launch.cuh"

namespace dilbm {

template <>
cudaError_t launch_step_sweep<__nv_bfloat16>(const SweepArgs<__nv_bfloat16> &a, bool edges, const SweepShape &sh, int num_sms,
                                   cudaStream_t st, bool query, int *per_sm) {
    return step_sweep_impl<__nv_bfloat16>(a, edges, sh, num_sms, st, query, per_sm);
}

template <>
cudaError_t launch_batch_sweep<__nv_bfloat16>(const BatchArgs<__nv_bfloat16> &ba, const SweepShape &sh, int num_sms, cudaStream_t st,
                                    bool query, int *per_sm) {
    return batch_sweep_impl<__nv_bfloat16>(ba, sh, num_sms, st, query, per_sm);
}

template <>
cudaError_t launch_step_sweep_ps<__nv_bfloat16>(const SweepArgs<__nv_bfloat16> &a, bool edges, int num_sms, cudaStream_t st) {
    return edges ? ps_variant<__nv_bfloat16, true>(a, num_sms, st) : ps_variant<__nv_bfloat16, false>(a, num_sms, st);
}

}  // namespace dilbm
