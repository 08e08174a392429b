// Host-side internals shared by the translation units of libgq (not part of
// the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gq.h"

// Per-thread record sizes (bytes, one or more 128-byte lines).
constexpr uint64_t kWfqRecBytes = 128;
constexpr uint64_t kYmcRecBytes = 128;
constexpr uint64_t kLine = 128;
// Distance between control lines.  Lines 128 or 256 bytes apart can share an
// L2 slice, and a slice serialises the atomics on its lines: two hot counters
// in one slice give the throughput of one.  4 KB apart they land in different
// slices (measured on GB300: same-address fetch-add throughput adds up over
// counters 4 KB apart, not over counters 128 B apart).
constexpr uint64_t kCtlStride = 4096;

struct gq_layout {
    uint64_t ctrl;       // control lines (error word, scratch, counters, thresholds)
    uint64_t aq_slots, fq_slots, data;
    uint64_t aq_rec, fq_rec, aq_owner, fq_owner, aq_helpc, fq_helpc;
    uint64_t cell_val, cell_enq, cell_deq, ymc_rec;
    uint64_t total;
};

// Control-region line indices.
enum {
    kCtlErr = 0,
    kCtlScratch = 1,
    kCtlAqHead = 2, kCtlAqTail = 3, kCtlAqThr = 4,
    kCtlFqHead = 5, kCtlFqTail = 6, kCtlFqThr = 7,
    kCtlYmcTail = 8, kCtlYmcHead = 9,
    kCtlAqSlow = 10, kCtlFqSlow = 11,
    kCtlYmcHw = 12,
    kCtlLines = 16
};

struct gq_queue {
    gq_dev dev;
    gq_layout lay;
    gq_options opt;
    void* ws;
    bool owned;
    int device;
    int sm_count;
    int smem_per_sm, smem_reserved, smem_optin;   // shared memory per SM, reserved per block, per-block maximum
    uint64_t start_ticket;
    void* aux;            // library-owned device scratch of the applications (gq_bfs), made on first use
    uint64_t aux_bytes;
    bool ymc_pool_known = false;   // G-WFQ-YMC: T, H and the scan mark bound the used cells (after the first reset)
};

// Status helpers
int gq_check_launch();

// Once per device (gq_create calls it, outside any stream capture): lets the
// G-LFQ run kernels take dynamic shared memory up to the per-block maximum, so
// that their residency-capped launches need no attribute call later (a launch
// being captured into a CUDA graph then makes none).
int gq_run_kernels_init(int device, int smem_optin);

// Threads of one gq_bfs launch of this queue kind on the current device (its
// cooperative grid: every resident 256-thread block); a G-WFQ / G-WFQ-YMC pair
// of frontier queues needs that many per-thread records.
int gq_bfs_grid_threads(int kind, uint64_t* threads);

// Launch configuration for a grid-stride kernel whose threads need one record
// each (G-WFQ, G-WFQ-YMC): never more threads than records.
void gq_grid_for(const gq_queue* q, uint64_t n_items, int occupancy_blocks_per_sm, uint32_t block,
                 uint32_t* grid_out);
