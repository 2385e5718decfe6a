// kernels.cuh -- launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tetproj_internal.h"

namespace tp {

enum { MODE_FWD = 0, MODE_BWD = 1, MODE_TRACE = 2 };

// One deferred ray: where its walk stopped, so the robust kernel continues
// from there.  fs < 0: deferred during the entry search (no state yet);
// otherwise fs = f | clip0 << 2 | steps << 3.
struct __align__(16) QEntry {
    int64_t ray;
    int32_t h;
    int32_t fs;
    float4 x;     // entry point of tet h (xyz); w = trace visits so far (int bits)
    float4 acc;   // forward partial sums (channels)
    float4 comp;  // their Kahan compensations
};
static_assert(sizeof(QEntry) == 64, "QEntry must be 64 bytes");

struct KParams {
    MeshView m;
    // ray source: cone-beam tiles (src_kind 0) or explicit rays (1)
    int32_t src_kind;
    GeoView g;
    const double *rsrc;
    const double *rdst;
    int64_t nrays;
    // ray tiles
    int32_t tu, tv, log_tu, log_tv, tiles_u, tiles_v, morton;
    // operands (Hilbert-ordered tet data; ray-ordered projection data)
    const void *in;   // FWD: mu_h [nt][C]; BWD: y [nrays][C]
    void *out;        // FWD: proj [nrays][C]; BWD: acc_h [nt][C]
    // trace outputs
    int32_t *tr_tet;
    double *tr_len;
    int32_t *tr_count;
    int32_t max_visits;
    int32_t max_steps;
    int32_t scatter;
    int32_t smem_nodes;
    // chunked launches: first block (cone tiles) or first block of 128 rays
    int64_t block_offset;
    // deferral queue of the filtered path (rays whose predicates the FP32
    // filter could not decide, with the walk state to continue from);
    // capacity >= rays per launch chunk
    struct QEntry *q;
    unsigned long long *q_count;
    int64_t q_cap;
    // OR-ed into the ray index of queue entries (batched launches: the problem
    // index in bits 40+; 0 otherwise)
    int64_t qtag;
};

// One problem of a batched launch: its parameters (operands included) and a
// spare 16 bytes so the 16-byte-vector copy into shared memory stays in bounds.
struct __align__(16) BatchProblem {
    KParams p;
    int64_t spare[2];
};

// Warp items per work chunk of the batched walk; every problem's item range
// starts at a multiple of it (a whole number of tiles of up to 256 rays).
constexpr int kBatchChunk = 8;

// Batched filtered walk over `nitems` warp items (32 rays of one tile) of
// `nprob` problems (problem k owns items [item_begin[k], item_begin[k+1]),
// item_begin[k] a multiple of kBatchChunk), in
// rounds of at most q_cap rays: per round one persistent work-queue launch of
// `grid` CTAs and one resume launch of `rgrid` CTAs.  `smem_nodes`: BVH nodes
// staged per warp.  Only stream operations (graph-capturable).
cudaError_t launch_batch(const BatchProblem *probs, const int64_t *item_begin, int nprob,
                         int64_t nitems, int channels, int mode, unsigned grid, unsigned rgrid,
                         QEntry *q, unsigned long long *q_count, int64_t q_cap,
                         unsigned *item_counter, int smem_nodes, cudaStream_t stream);
// Persistent grid for the batched walk: resident CTAs per SM x SM count.
cudaError_t batch_grid(int channels, int mode, int smem_nodes, unsigned &grid);
int device_sm_count();

// one launch of the walk; returns a cudaError_t
cudaError_t launch_walk(const KParams &p, int precision, int channels, int mode,
                        cudaStream_t stream);
cudaError_t launch_gather_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                               const void *src_user, void *dst_h, cudaStream_t stream);
cudaError_t launch_scatter_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                                const void *src_h, void *dst_user, cudaStream_t stream);
cudaError_t launch_geometry_rays(const GeoView &g, const int64_t *idx, int64_t n, double *src,
                                 double *dst, cudaStream_t stream);
cudaError_t launch_side_device(const double *S, const double *P, const double *p,
                               const double *q, int64_t n, int8_t *sign, int8_t *stage,
                               cudaStream_t stream);

}  // namespace tp
