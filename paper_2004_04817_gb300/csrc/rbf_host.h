// rbf_host.h -- host-side helpers of librbfgcb (device queries, workspace
// arithmetic, the seeded partition generator).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rbfgcb.h"

namespace rbf {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DeviceInfo {
    int device;
    int sms;
    int coop;          // cooperative launch supported
    size_t smem_optin; // max dynamic shared memory per block
};

// Queries (and caches per device) the current device's properties.
bool device_info(DeviceInfo *out);

// True when the device can read and write p at that address: device or
// managed memory, or pinned host memory mapped at the same address.
bool device_accessible(const void *p);

// Grid barrier wait limit for the persistent kernels.
constexpr uint64_t kBarrierLimitNs = 4000000000ull;   // 4 s

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) -- one step of the stream.
inline uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Random permutation of 0..n-1: Fisher-Yates from the last position down,
// position i swapped with j = next() mod (i + 1).  Node perm[p] is put in group
// p mod m by the greedy (Sec. 3: disjoint groups whose sizes differ by <= 1).
void fisher_yates(int64_t n, uint64_t seed, int32_t *perm);

}  // namespace rbf

// A factorised support system (rbf_factor_*): the caller-owned arrays it was
// made from and its workspace, which holds Z = L^-1 of Phi_SS.
struct rbf_factor {
    const double *xb;
    int64_t nb;
    const int32_t *sel;
    int64_t nc;
    double radius;
    char *ws;
    size_t ws_bytes;
};
