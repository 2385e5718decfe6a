// kernels.cuh -- launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tetproj_internal.h"

namespace tp {

// MODE_SEG: the backprojection's sort-and-reduce variant -- the walk writes
// each segment (tet, length x y) to a segment buffer instead of adding it.
// MODE_ENTRY: only the entry search; the entry tet's user id (or -1) goes to
// tr_count[ray].  MODE_BWD64: the filtered backprojection with FP64
// accumulation (p.out is a double [nt][C] buffer; red.global.add.f64).
enum { MODE_FWD = 0, MODE_BWD = 1, MODE_TRACE = 2, MODE_SEG = 3, MODE_ENTRY = 4, MODE_BWD64 = 5 };
// entry-search structure of the fast walk
enum { ENTRY_BVH = 0, ENTRY_RSTAR = 1 };

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

// A crossing the fast walk placed in FP32 although the ray meets the face at a
// grazing angle (FP32 vertex rounding moves such a crossing by ~u|v|/sin along
// the ray): the correction kernel places it again from the FP64 records and
// moves the difference between the two segments that meet there (a ray's
// integral is linear in each crossing's position along it).
struct __align__(16) XFix {
    int64_t ray;    // ray index (| qtag in batched launches)
    int32_t h;      // tet the crossing leaves
    int32_t hn;     // tet it enters, or -1 (the ray leaves the mesh)
    float x, y, z;  // the FP32 crossing the walk used
    int32_t fx;     // entry face of h | exit index << 2
};
static_assert(sizeof(XFix) == 32, "XFix must be 32 bytes");

// A deferral queue's allocation also holds the crossing fixes of the same
// launch chunk: q[0 .. cap) QEntry, then (cap / 2) XFix; its count words are
// q_count[0] (deferred rays) and q_count[1] (fixes).  A walk that finds the
// fix list full defers the ray instead (the resume walk places crossings in
// FP64 itself).
inline int64_t queue_bytes(int64_t cap) {
    return cap * (int64_t)sizeof(QEntry) + (cap / 2) * (int64_t)sizeof(XFix);
}
constexpr size_t kQueueCountBytes = 2 * sizeof(unsigned long long);
__host__ __device__ inline XFix *queue_fixes(QEntry *q, int64_t cap) {
    return reinterpret_cast<XFix *>(q + cap);
}

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
    // MODE_SEG (cone rays only): segment j of ray r (tile block b) goes to
    // slot s = block_off[b] - seg_base + ray_off[r] + j, s in [0, seg_cap):
    // C = 1: uint2 (tet, value bits) at ((uint2 *)seg_key)[s]; C = 4: the tet
    // at seg_key[s] and a float4 at ((float4 *)seg_val)[s]
    uint32_t *seg_key;
    float *seg_val;
    const int64_t *block_off;
    const int32_t *ray_off;
    int64_t seg_base, seg_cap;
    int32_t entry;  // ENTRY_BVH or ENTRY_RSTAR (fast walk, FWD C = 1 and ENTRY modes)
    // Candidate entry faces of cone rays (fast walk, BVH entry): when emap_buf
    // is set, each launch chunk first draws the boundary faces its angles'
    // sources see from outside onto the detector (k_entry_raster), so that
    // emap[ray - emap_base] (0 <= . < emap_len) is a boundary face whose
    // projection covers the ray's pixel, or -1.  The walk tests that face with
    // its exact entry test and searches the BVH only when it is not the one.
    int32_t *emap_buf;   // emap_cap ints, or null (no map)
    int64_t emap_cap;
    const int32_t *emap;
    int64_t emap_base, emap_len;
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
// staged per warp.  With `ov` (its q2 holding q_cap entries) and more than one
// round, round r's resume runs on ov->aux beside round r + 1's walk.  Rounds
// hold at most q_cap rays: uniform, or the item ranges [cuts[i], cuts[i + 1])
// (cuts[0] = 0, cuts[ncuts - 1] = nitems); after each round's resume the
// `nmerge` accumulator merges run (MODE_BWD).  Only stream and event
// operations (graph-capturable).
struct ResumeOverlap;
struct AccMerge;
// Warp items per uniform round of the batched launch (rounds hold at most
// q_cap rays and whole work chunks).
inline int64_t batch_round_items(int64_t q_cap) {
    return (q_cap / (32 * kBatchChunk)) * kBatchChunk;
}
// Entry map of one problem in one round of the batched launch (see
// KParams::emap): emap[ray - base], 0 <= . < len, or emap == null.
struct EmapView {
    const int32_t *emap;
    int64_t base, len;
};
// The rasters of one round: problem `prob`'s angles [a_lo, a_lo + na) drawn
// into buf + off; rounds list their jobs [first, first + count) and the
// length (ints) of the buffer they use.
struct BatchEmapJob {
    int32_t prob, a_lo, na;
    int64_t off;
};
struct BatchEmapRound {
    int32_t first, count;
    int64_t len;
};
struct BatchEmap {
    int32_t *buf;                  // device, shared by the rounds (one at a time)
    const EmapView *views;         // device [nrounds][nprob]: the rounds' views
    const BatchEmapRound *rounds;  // host [nrounds]
    const BatchEmapJob *jobs;      // host
    const KParams *probs;          // host [nprob]: mesh and geometry of each problem
    int nprob;
};
// The bounded waits between the warps of a batched CTA: at most `limit` polls
// each (kBatchWaitPolls by default), then TETPROJ_ERR_TIMEOUT and the warp
// stops.  A non-zero `offset` makes every wait wait for a value no warp
// writes (a test of the timeout path).
struct BatchWait {
    int limit;
    int offset;
};
constexpr int kBatchWaitPolls = 1 << 22;
cudaError_t launch_batch(const BatchProblem *probs, const int64_t *item_begin, int nprob,
                         int64_t nitems, int channels, int mode, unsigned grid, unsigned rgrid,
                         QEntry *q, unsigned long long *q_count, int64_t q_cap,
                         unsigned *item_counter, int smem_nodes, cudaStream_t stream,
                         const ResumeOverlap *ov, const int64_t *cuts, int ncuts,
                         const AccMerge *merges, int nmerge, BatchWait wait,
                         const BatchEmap *emap = nullptr);
// Persistent grid for the batched walk: resident CTAs per SM x SM count.
cudaError_t batch_grid(int channels, int mode, int smem_nodes, unsigned &grid);
int device_sm_count();

// Filtered walk over the tile blocks [b0, b1) (b1 - b0 <= q_cap / threads):
// one fast and one resume launch.  Cone rays; modes FWD, BWD, TRACE, SEG.
cudaError_t launch_walk_blocks(const KParams &p, int channels, int mode, int64_t b0, int64_t b1,
                               cudaStream_t stream);
// Per tile block b: ray_off[r] = exclusive prefix of max(count[r], 0) over the
// block's rays in thread order, block_cnt[b] = their sum (cone rays).
cudaError_t launch_block_offsets(const KParams &p, const int32_t *count, int32_t *ray_off,
                                 int64_t *block_cnt, int64_t nblocks, cudaStream_t stream);
// Exclusive prefix sums out[0..n] of in[0..n-1] (out[n] = total); `tmp` holds
// scan_temp_elems(n) elements.
int64_t scan_temp_elems(int64_t n);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                            cudaStream_t stream);
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                            cudaStream_t stream);
// Stable LSD radix sort of n segment records by the low `key_bits` bits of
// the key (8 bits per pass).  Records: C = 1, uint2 (key, value bits) in the k
// buffers (v unused); C = 4, keys in k and float4 values in v.  Sorted data
// ends in (*k_out, *v_out), either the a or the b buffers.  `hist` holds
// radix_hist_elems(n) and `tmp` scan_temp_elems(radix_hist_elems(n)) words.
int64_t radix_hist_elems(int64_t n);
cudaError_t launch_radix_sort(uint32_t *k_a, float *v_a, uint32_t *k_b, float *v_b, int64_t n,
                              int channels, int key_bits, uint32_t *hist, uint32_t *tmp,
                              uint32_t **k_out, float **v_out, cudaStream_t stream);
// acc[key][c] += sum of each run of equal keys of the sorted records (Kahan,
// in order): deterministic.  scratch: seg_reduce_scratch_elems(n) words; tmp:
// scan_temp_elems(n) words.
int64_t seg_reduce_scratch_elems(int64_t n);
cudaError_t launch_seg_reduce(const uint32_t *keys, const float *vals, int64_t n, int channels,
                              float *acc, uint32_t *scratch, uint32_t *tmp, cudaStream_t stream);

// Host-side count of the kernels this library has launched (every launcher
// calls note_launch once per launch; graph replays are not seen).
void note_launch();
long long launch_count();

// The paper's own walk (Alg. 1 and 2, Moller-Trumbore with a growing safety
// margin) in FP32 (f64 = 0) or FP64: C = 1 forward into p.out, per-ray
// status 0 done / 1 halted (no two faces found) / 2 step limit; tiles of at
// most 128 threads.
cudaError_t launch_walk_mt(const KParams &p, int f64, int8_t *status, cudaStream_t stream);

// Second deferral queue and an auxiliary stream: with them a filtered walk of
// several chunks runs each chunk's resume kernel on `aux` while the next
// chunk's fast kernel runs on the caller's stream (queues alternate; events
// order each queue's reuse and join `aux` back before the call returns).
struct ResumeOverlap {
    QEntry *q2;
    unsigned long long *q2_count;
    cudaStream_t aux;
    cudaEvent_t ev_fast[2], ev_res[2], ev_start;
};

// Two-level accumulation of the FP32 backprojection: the walk reduces into
// acc32 (FP32, n floats) and, after each chunk of at most chunk_rays rays
// (and its resume kernel), acc32 is moved into acc64 and zeroed, so that no
// FP32 sum collects more than one chunk's contributions.  The move reads
// acc32 with atomic exchanges: reductions of a chunk running at the same time
// (overlapped resume) land either before or after it and are never lost.
struct AccMerge {
    float *acc32;
    double *acc64;
    int64_t n;
    int64_t chunk_rays;
};
cudaError_t launch_acc_merge(float *acc32, double *acc64, int64_t n, cudaStream_t stream);

// one launch of the walk; returns a cudaError_t.  `mg` (MODE_BWD only): the
// walk's p.out is mg->acc32, merged into mg->acc64 after every chunk.
cudaError_t launch_walk(const KParams &p, int precision, int channels, int mode,
                        cudaStream_t stream, const ResumeOverlap *ov = nullptr,
                        const AccMerge *mg = nullptr);
cudaError_t launch_gather_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                               const void *src_user, void *dst_h, cudaStream_t stream);
cudaError_t launch_scatter_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                                const void *src_h, void *dst_user, cudaStream_t stream);
// the same from a double accumulator into float output (rounded once)
cudaError_t launch_scatter_perm_d2f(const int32_t *perm, int64_t nt, int channels,
                                    const double *src_h, float *dst_user, cudaStream_t stream);
cudaError_t launch_geometry_rays(const GeoView &g, const int64_t *idx, int64_t n, double *src,
                                 double *dst, cudaStream_t stream);
cudaError_t launch_side_device(const double *S, const double *P, const double *p,
                               const double *q, int64_t n, int8_t *sign, int8_t *stage,
                               cudaStream_t stream);

}  // namespace tp
