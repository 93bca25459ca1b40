// Dispatch of the temporally blocked kernels by polarisation; the
// instances live in blocked_s.cu, blocked_sb.cu and blocked_p.cu (compiled
// in parallel), the kernel templates in blocked_impl.cuh.
#include "blocked_impl.cuh"

namespace fdtd {

int blocked_max_K() { return 8; }

int blocked_warps_per_sm(int K, int variant, int pol) {
    return pol ? blocked_occupancy_p(K, variant) : blocked_occupancy_s(K, variant);
}

bool launch_blocked(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st) {
    return a.s.pol ? launch_blocked_p(a, K, variant, n0, st) : launch_blocked_s(a, K, variant, n0, st);
}

bool launch_blocked_batch(const BatchArgs& b, int K, int variant, int step_off, int parity,
                          int pol, cudaStream_t st) {
    return pol ? launch_blocked_batch_p(b, K, variant, step_off, parity, st)
               : launch_blocked_batch_s(b, K, variant, step_off, parity, st);
}

}  // namespace fdtd
