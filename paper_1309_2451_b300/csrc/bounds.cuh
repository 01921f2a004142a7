// bounds.cuh -- the bounds-checked build (CTAP_DEBUG_BOUNDS).
//
// Compiled with -DCTAP_DEBUG_BOUNDS, every index the checked kernels use
// for a shared-memory or HBM access is compared with the extent of its
// buffer first.  A violation never traps: the first one is recorded in a
// device word of the including file (check site in the top 16 bits, the
// offending index below) and the access is skipped, so the context stays
// usable and the host reads the record with ctap_debug_bounds.  In the
// normal build the check is the constant true and costs nothing.
#pragma once

#ifdef CTAP_DEBUG_BOUNDS
static __device__ unsigned long long g_ctap_bounds = 0;
__device__ __forceinline__ bool ctap_in_bounds(int site, long long idx, long long lim)
{
    if (idx >= 0 && idx < lim) return true;
    atomicCAS(&g_ctap_bounds, 0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xffffffffffffull));
    return false;
}
#define CTAP_BOUNDS(site, idx, lim) ctap_in_bounds((site), (long long)(idx), (long long)(lim))
#else
#define CTAP_BOUNDS(site, idx, lim) true
#endif
