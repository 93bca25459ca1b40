// S-polarised (TMz) instances of the blocked kernel for single runs: code
// shapes 0-6 at K = 1..8 (shapes 4 and 6 serve the adjoint's recompute,
// shapes 5 and 6 handles with at most 16 labels).
#include "blocked_impl.cuh"

namespace fdtd {

int blocked_occupancy_s(int K, int variant) {
    switch (K) {
#define X(k)                                                                   \
    case k:                                                                    \
        if (variant == 3) return occupancy_of(k_blocked_cap<k, 0>);            \
        if (variant == 4) return occupancy_of(k_blocked<k, 4, 0>);             \
        if (variant == 5) return occupancy_of(k_blocked<k, 5, 0>);             \
        if (variant == 6) return occupancy_of(k_blocked<k, 6, 0>);             \
        if (variant == 2) return occupancy_of(k_blocked<k, 2, 0>);             \
        return variant ? occupancy_of(k_blocked<k, 1, 0>) : occupancy_of(k_blocked<k, 0, 0>);
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return 0;
    }
}

bool launch_blocked_s(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st) {
    const unsigned grid = (unsigned)a.n_tasks;
    switch (K) {
#define X(k)                                                                   \
    case k:                                                                    \
        if (variant == 3) k_blocked_cap<k, 0><<<grid, 32, 0, st>>>(a, n0);     \
        else if (variant == 4) k_blocked<k, 4, 0><<<grid, 32, 0, st>>>(a, n0); \
        else if (variant == 5) k_blocked<k, 5, 0><<<grid, 32, 0, st>>>(a, n0); \
        else if (variant == 6) k_blocked<k, 6, 0><<<grid, 32, 0, st>>>(a, n0); \
        else if (variant == 2) k_blocked<k, 2, 0><<<grid, 32, 0, st>>>(a, n0); \
        else if (variant) k_blocked<k, 1, 0><<<grid, 32, 0, st>>>(a, n0);      \
        else k_blocked<k, 0, 0><<<grid, 32, 0, st>>>(a, n0);                   \
        break;
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return false;
    }
    return true;
}

}  // namespace fdtd
