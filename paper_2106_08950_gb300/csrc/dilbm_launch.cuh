// Launch shapes of the lattice sweep and the launchers that take them.
//
// A shape is numerics-neutral: it only decides how many row segments a block
// keeps in flight (warps per block, one row segment per warp) and how many
// blocks the persistent grid holds per SM.  Every node is swept by the same
// code in the same arithmetic whatever the shape, so the autotuner may pick
// any shape without changing a single result bit.
//
// The launchers of the step sweep are compiled once per storage type, each
// in its own translation unit (dilbm_launch_f32.cu, _f16.cu, _bf16.cu).
#pragma once
#include "dilbm_kernels.cuh"

namespace dilbm {

struct SweepShape {
    int warps = SWEEP_WARPS;    // rows in flight per block: 2, 4 or 8
    int blocks_per_sm = 0;      // persistent blocks per SM; 0: as many as fit
};

constexpr int SHAPE_WARPS[3] = {2, 4, 8};

__host__ inline bool shape_valid(const SweepShape &s) {
    return (s.warps == 2 || s.warps == 4 || s.warps == 8) && s.blocks_per_sm >= 0;
}

// Blocks of `kern` (W warps, `smem` bytes of dynamic shared memory) resident
// per SM, after opting in to that shared memory; cached per device.
template <typename K>
cudaError_t occupancy_of(K kern, int warps, size_t smem, int *cache, int *per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (cache[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, warps * 32, smem);
        if (e != cudaSuccess) return e;
        cache[dev] = n > 0 ? n : 1;
    }
    *per_sm = cache[dev];
    return cudaSuccess;
}

// Persistent grid: num_sms x blocks per SM (capped by the shape and by the
// kernel's occupancy), but no more blocks than the row segments need.
inline long long persistent_grid(long long items, int warps, int per_sm, int num_sms, const SweepShape &sh) {
    const int bps = sh.blocks_per_sm > 0 && sh.blocks_per_sm < per_sm ? sh.blocks_per_sm : per_sm;
    long long blocks = (long long)num_sms * bps;
    const long long need = (items + warps - 1) / warps;
    if (blocks > need) blocks = need;
    return blocks > 0 ? blocks : 1;
}

template <typename T, bool EDGES, int W>
cudaError_t step_variant(const SweepArgs<T> &a, const SweepShape &sh, int num_sms, cudaStream_t st, bool query,
                         int *per_sm_out) {
    static int cache[64] = {};
    constexpr size_t smem = sweep_smem_bytes<T, W>();
    int per_sm = 1;
    cudaError_t e = occupancy_of(sweep_kernel<T, MODE_STEP, EDGES, W>, W, smem, cache, &per_sm);
    if (e != cudaSuccess || query) {
        if (per_sm_out) *per_sm_out = per_sm;
        return e;
    }
    const long long items = (long long)a.L.ny * a.L.ntx;
    const long long blocks = persistent_grid(items, W, per_sm, num_sms, sh);
    sweep_kernel<T, MODE_STEP, EDGES, W><<<(unsigned)blocks, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t batch_variant(const BatchArgs<T> &ba, const SweepShape &sh, int num_sms, cudaStream_t st, bool query,
                          int *per_sm_out) {
    static int cache[64] = {};
    constexpr size_t smem = sweep_smem_bytes<T, W>();
    int per_sm = 1;
    cudaError_t e = occupancy_of(sweep_batch_kernel<T, MODE_STEP, W>, W, smem, cache, &per_sm);
    if (e != cudaSuccess || query) {
        if (per_sm_out) *per_sm_out = per_sm;
        return e;
    }
    const long long blocks = persistent_grid(ba.item_start[ba.n], W, per_sm, num_sms, sh);
    sweep_batch_kernel<T, MODE_STEP, W><<<(unsigned)blocks, W * 32, smem, st>>>(ba);
    return cudaGetLastError();
}

// The PS-LBM step sweep (the paper's comparison method), in the default shape.
template <typename T, bool EDGES>
cudaError_t ps_variant(const SweepArgs<T> &a, int num_sms, cudaStream_t st) {
    static int cache[64] = {};
    constexpr size_t smem = sweep_smem_bytes<T>();
    int per_sm = 1;
    cudaError_t e = occupancy_of(sweep_kernel<T, MODE_STEP, EDGES, SWEEP_WARPS, true>, SWEEP_WARPS, smem, cache, &per_sm);
    if (e != cudaSuccess) return e;
    const long long blocks = persistent_grid((long long)a.L.ny * a.L.ntx, SWEEP_WARPS, per_sm, num_sms, SweepShape{});
    sweep_kernel<T, MODE_STEP, EDGES, SWEEP_WARPS, true><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// Generic bodies of the per-storage launchers.
template <typename T>
cudaError_t step_sweep_impl(const SweepArgs<T> &a, bool edges, const SweepShape &sh, int num_sms, cudaStream_t st,
                            bool query, int *per_sm) {
    switch (sh.warps) {
    case 2: return edges ? step_variant<T, true, 2>(a, sh, num_sms, st, query, per_sm)
                         : step_variant<T, false, 2>(a, sh, num_sms, st, query, per_sm);
    case 4: return edges ? step_variant<T, true, 4>(a, sh, num_sms, st, query, per_sm)
                         : step_variant<T, false, 4>(a, sh, num_sms, st, query, per_sm);
    case 8: return edges ? step_variant<T, true, 8>(a, sh, num_sms, st, query, per_sm)
                         : step_variant<T, false, 8>(a, sh, num_sms, st, query, per_sm);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t batch_sweep_impl(const BatchArgs<T> &ba, const SweepShape &sh, int num_sms, cudaStream_t st, bool query,
                             int *per_sm) {
    switch (sh.warps) {
    case 2: return batch_variant<T, 2>(ba, sh, num_sms, st, query, per_sm);
    case 4: return batch_variant<T, 4>(ba, sh, num_sms, st, query, per_sm);
    case 8: return batch_variant<T, 8>(ba, sh, num_sms, st, query, per_sm);
    default: return cudaErrorInvalidValue;
    }
}

// Per-storage launchers (defined in dilbm_launch_f32.cu, _f16.cu, _bf16.cu).
// query != 0: launch nothing, return the kernel's resident blocks per SM in
// *per_sm.
template <typename T>
cudaError_t launch_step_sweep(const SweepArgs<T> &a, bool edges, const SweepShape &sh, int num_sms, cudaStream_t st,
                              bool query = false, int *per_sm = nullptr);
template <typename T>
cudaError_t launch_batch_sweep(const BatchArgs<T> &ba, const SweepShape &sh, int num_sms, cudaStream_t st,
                               bool query = false, int *per_sm = nullptr);

template <> cudaError_t launch_step_sweep<float>(const SweepArgs<float> &, bool, const SweepShape &, int, cudaStream_t, bool, int *);
template <> cudaError_t launch_step_sweep<__half>(const SweepArgs<__half> &, bool, const SweepShape &, int, cudaStream_t, bool, int *);
template <> cudaError_t launch_step_sweep<__nv_bfloat16>(const SweepArgs<__nv_bfloat16> &, bool, const SweepShape &, int, cudaStream_t, bool, int *);
template <typename T>
cudaError_t launch_step_sweep_ps(const SweepArgs<T> &a, bool edges, int num_sms, cudaStream_t st);
template <> cudaError_t launch_step_sweep_ps<float>(const SweepArgs<float> &, bool, int, cudaStream_t);
template <> cudaError_t launch_step_sweep_ps<__half>(const SweepArgs<__half> &, bool, int, cudaStream_t);
template <> cudaError_t launch_step_sweep_ps<__nv_bfloat16>(const SweepArgs<__nv_bfloat16> &, bool, int, cudaStream_t);
template <> cudaError_t launch_batch_sweep<float>(const BatchArgs<float> &, const SweepShape &, int, cudaStream_t, bool, int *);
template <> cudaError_t launch_batch_sweep<__half>(const BatchArgs<__half> &, const SweepShape &, int, cudaStream_t, bool, int *);
template <> cudaError_t launch_batch_sweep<__nv_bfloat16>(const BatchArgs<__nv_bfloat16> &, const SweepShape &, int, cudaStream_t, bool, int *);

}  // namespace dilbm
