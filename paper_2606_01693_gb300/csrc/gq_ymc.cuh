// G-WFQ-YMC (Section III-A).  Placeholder until it lands.
#pragma once
#include "gq_atomics.cuh"
namespace gqd {
template <class T, bool MATCH>
__device__ int ymc_enqueue(const gq_dev& q, T v, u32 tid) { return GQ_ERR_INVALID; }
template <class T, bool MATCH>
__device__ int ymc_dequeue(const gq_dev& q, T* v, u32 tid) { return GQ_ERR_INVALID; }
}  // namespace gqd
