// A user kernel built against the public device API only (include/gq_device.cuh),
// as a library user would: compiled by the device-API test into its own shared
// object.  Thread i of `n` (n even) enqueues in[i / 2] if i is even -- from one
// of two call sites chosen by the value's low bit, so the lanes that reach each
// call are a divergent subset -- and dequeues one item into out[i / 2] if i is
// odd, retrying on EMPTY (a bounded number of times).
#include <cuda_runtime.h>

#include "gq_device.cuh"

__global__ void user_mixed(const __grid_constant__ gq_dev q, const unsigned long long* in, unsigned long long* out,
                           int* status, unsigned n) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s;
    if ((i & 1) == 0) {
        const unsigned long long v = in[i / 2];
        if (v & 1) s = gq_enqueue(q, v, i);
        else s = gq_enqueue(q, v, i);
    } else {
        unsigned long long v = 0;
        s = GQ_EMPTY;
        for (int a = 0; a < (1 << 20) && s == GQ_EMPTY; ++a) {
            s = gq_dequeue(q, &v, i);
            if (s == GQ_EMPTY) __nanosleep(100);
        }
        out[i / 2] = v;
    }
    status[i] = s;
}

extern "C" int user_mixed_launch(const void* view, const unsigned long long* in, unsigned long long* out, int* status,
                                 unsigned n) {
    gq_dev q;
    memcpy(&q, view, sizeof(q));
    user_mixed<<<(n + 255) / 256, 256>>>(q, in, out, status, n);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
