// The filter handle behind the C ABI (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/blowchoc.h"
#include "bc_device.cuh"

struct blowchoc_filter {
    blowchoc_params p;
    bc::DevFilter dev;             // words pointer, M, k, hash parameters
    uint16_t *d_rank = nullptr;    // 513 x (k+1) cost ranks (c > 1)
    unsigned long long *d_counters = nullptr;  // [0] inserted [1] skipped [2] error [3..515] hist
                                               // [516] grid-barrier arrivals (u32)
    uint8_t *d_sel = nullptr;      // per-key choices of one batch
    uint64_t sel_cap = 0;
    cudaStream_t home = nullptr;
    int device = 0;
    int sms = 0;
    int lanes_choose = 2, lanes_set = 4, lanes_query = 2;
    int query_early = 1;
    int ctas_per_sm = 8;
    int persistent = 1;            // insert: one cooperative launch for all batches
    int keys_per_cta = 128;        // persistent insert grid: keys of a batch per CTA
    int set_mode = 0;              // 0: atomic OR at L2; 1: sort by block range
    uint32_t *d_sorted = nullptr;  // sort-by-block scratch (3 R + 1 + batch u32)
    uint64_t sorted_cap = 0;
    int seq_window = 512;          // B <= 16: keys per reservation window, set at creation (0: one-warp kernel)
    unsigned long long *d_resv = nullptr;  // B = 1 reservations, M words
    int cluster_max = 16;          // cluster-resident insert: CTAs per cluster at most (0: off)
    int lanes_cluster = 8;
    int cluster_keys = 128;        // keys of a batch per CTA the cluster size aims for
    uint32_t host_ring_keys = 0;   // host-buffer staging ring limit in keys (0: the default)
    struct HostStage *host = nullptr;  // host-buffer calls' staging (bc_host.cu), made on first use
};

// Frees the host-buffer staging of f (synchronises its copy stream).
void bc_free_host_stage(blowchoc_filter *f);

// Adds one to the library's launch counter (blowchoc_launch_count).
void bc_note_launch();

// Records msg as the calling thread's last error (blowchoc_last_error); returns code.
int bc_set_error(int code, const char *msg);

// Allocates the device scratch that blowchoc_insert of n keys into f would
// allocate on first use, without launching (for graph capture).
extern "C" int bc_reserve_insert_scratch(blowchoc_filter *f, uint64_t n);

// Checks the fields of a filter launch configuration; EINVAL with a message.
extern "C" int bc_check_tuning(const blowchoc_tuning *t);
