// Step-sweep and batched-sweep launchers for float storage, every launch
// shape (warps per block 2, 4, 8; with and without edge handling).  One
// translation unit per storage type so that the library compiles in parallel.
#include "dilbm_launch.cuh"

namespace dilbm {

template <>
cudaError_t launch_step_sweep<float>(const SweepArgs<float> &a, bool edges, const SweepShape &sh, int num_sms,
                                   cudaStream_t st, bool query, int *per_sm) {
    return step_sweep_impl<float>(a, edges, sh, num_sms, st, query, per_sm);
}

template <>
cudaError_t launch_batch_sweep<float>(const BatchArgs<float> &ba, const SweepShape &sh, int num_sms, cudaStream_t st,
                                    bool query, int *per_sm) {
    return batch_sweep_impl<float>(ba, sh, num_sms, st, query, per_sm);
}

template <>
cudaError_t launch_step_sweep_ps<float>(const SweepArgs<float> &a, bool edges, int num_sms, cudaStream_t st) {
    return edges ? ps_variant<float, true>(a, num_sms, st) : ps_variant<float, false>(a, num_sms, st);
}

}  // namespace dilbm
