// segsort.cu -- the sort-and-reduce variant of the backprojection scatter.
//
// The walk (MODE_SEG) writes every segment of a chunk of rays as a pair
// (tet h, length x y_ray) at a position fixed by the rays' segment counts, so
// the buffer's order depends only on the input.  A stable LSD radix sort by h
// (8-bit digits) groups the pairs of each tet in that same order, and one
// thread per run of equal keys sums the run sequentially.  Every addition
// happens in an order fixed by the input: the result is bit-reproducible, unlike
// the atomic scatters, whose order is the hardware's.  The paper adds with
// atomics (Sec. II-F); this is the alternative it is measured against.
//
// Also here: exclusive prefix sums (for the segment offsets and the radix
// histograms).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace tp {

#define SS_FULL 0xffffffffu

// ------------------------------------------------------------- prefix sums
//
// Three phases: each CTA scans SCAN_TILE elements and records its total;
// the totals are scanned (recursively); each CTA adds its total's prefix.

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(SS_FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// out[i] = exclusive prefix within the tile; sums[tile] = tile total
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_tiles(const T *__restrict__ in, T *__restrict__ out, int64_t n, T *__restrict__ sums) {
    __shared__ T wtot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : T(0);
        run += v[k];
    }
    const T incl = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    if (w == 0) {
        T t = lane < SCAN_THREADS / 32 ? wtot[lane] : T(0);
        T ti = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) wtot[lane] = ti - t;  // exclusive
    }
    __syncthreads();
    T pre = wtot[w] + incl - run;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = pre;  // tile total
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_add(T *__restrict__ out, int64_t n, const T *__restrict__ tile_pre) {
    const T add = tile_pre[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
        const int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

int64_t scan_temp_elems(int64_t n) {
    // tile totals and their prefixes at every level
    int64_t t = 0;
    while (n > 1) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        t += 2 * n + 2;
    }
    return t + 2;
}

// out[0..n-1] exclusive prefix, out[n] total.  tmp: scan_temp_elems(n) elements.
template <typename T>
static cudaError_t scan_rec(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(T), s);
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
    T *sums = tmp;             // tiles
    T *pre = tmp + tiles;      // tiles + 1
    k_scan_tiles<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (tiles == 1) {
        // the single tile's total is the grand total
        e = cudaMemcpyAsync(out + n, sums, sizeof(T), cudaMemcpyDeviceToDevice, s);
        return e;
    }
    e = scan_rec<T>(sums, pre, tiles, tmp + 2 * tiles + 2, s);
    if (e != cudaSuccess) return e;
    k_scan_add<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(out, n, pre);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(out + n, pre + tiles, sizeof(T), cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                            cudaStream_t stream) {
    return scan_rec<int64_t>(in, out, n, tmp, stream);
}

cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                            cudaStream_t stream) {
    return scan_rec<uint32_t>(in, out, n, tmp, stream);
}

// -------------------------------------------------------------- radix sort
//
// Segments are records: C = 1 packs (tet, value bits) into one uint2; C = 4
// keeps a key array and a float4 value array.  One pass sorts by the 8-bit
// digit d = (key >> shift) & 255, stably:
//   1. k_radix_hist: per tile, the digit histogram, stored digit-major
//      (hist[d * G + tile]);
//   2. exclusive scan of hist: the first output slot of (digit, tile);
//   3. k_radix_scatter: each warp ranks its 32-key rounds with
//      __match_any_sync (lanes with one digit, in lane order) on top of the
//      warp's running digit counts; warps own consecutive sub-tiles, so the
//      prefix of the warps' counts completes a stable rank within the tile.
//      The tile is first placed in digit order in shared memory, then copied
//      out in that order: consecutive threads write consecutive slots of one
//      digit's output range (coalesced), not 32 different ranges per store.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

template <int C> struct RsCfg;
template <> struct RsCfg<1> { static constexpr int ROUNDS = 16; };  // 4096 records, 32 KB
template <> struct RsCfg<4> { static constexpr int ROUNDS = 6; };   // 1536 records, 30 KB

int64_t radix_hist_elems(int64_t n) {
    // the smaller tile (C = 4) has the most tiles
    return 256 * ((n + RS_THREADS * RsCfg<4>::ROUNDS - 1) / (RS_THREADS * RsCfg<4>::ROUNDS)) + 1;
}

template <int C>
__device__ __forceinline__ uint32_t rs_key(const uint32_t *keys, int64_t i) {
    if (C == 1) return __ldg(reinterpret_cast<const uint2 *>(keys) + i).x;
    return __ldg(keys + i);
}

template <int C>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist,
                 int64_t G) {
    constexpr int TILE = RS_THREADS * RsCfg<C>::ROUNDS;
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * TILE;
    for (int k = threadIdx.x; k < TILE; k += RS_THREADS) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&h[(rs_key<C>(keys, i) >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * G + blockIdx.x] = h[threadIdx.x];
}

// block-wide exclusive scan of one value per thread (RS_THREADS = 256)
__device__ __forceinline__ uint32_t rs_block_excl(uint32_t x, uint32_t *wtmp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(x);
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < RS_WARPS ? wtmp[lane] : 0u;
        uint32_t ti = warp_incl_scan(t);
        if (lane < RS_WARPS) wtmp[lane] = ti - t;
    }
    __syncthreads();
    return wtmp[w] + incl - x;
}

template <int C>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_scatter(const uint32_t *__restrict__ kin, const float *__restrict__ vin,
                    uint32_t *__restrict__ kout, float *__restrict__ vout, int64_t n, int shift,
                    const uint32_t *__restrict__ offs, int64_t G) {
    constexpr int ROUNDS = RsCfg<C>::ROUNDS;
    constexpr int TILE = RS_THREADS * ROUNDS;
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t goff[256], toff[256], wtmp[RS_WARPS];
    // staging: C = 1 records (8 B), C = 4 keys then values (4 + 16 B)
    __shared__ __align__(16) unsigned char stage[C == 1 ? TILE * 8 : TILE * 20];
    uint2 *srec = reinterpret_cast<uint2 *>(stage);
    uint32_t *skey = reinterpret_cast<uint32_t *>(stage);
    float4 *sval = reinterpret_cast<float4 *>(stage + (C == 1 ? 0 : TILE * 4));

    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    goff[threadIdx.x] = __ldg(offs + (int64_t)threadIdx.x * G + blockIdx.x);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * TILE;
    const int64_t base = tile0 + (int64_t)w * (32 * ROUNDS);
    uint32_t key[ROUNDS], aux[ROUNDS], rank[ROUNDS];
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        if (C == 1) {
            const uint2 rec = valid ? __ldg(reinterpret_cast<const uint2 *>(kin) + i) : make_uint2(0u, 0u);
            key[r] = rec.x;
            aux[r] = rec.y;
        } else {
            key[r] = valid ? __ldg(kin + i) : 0u;
            aux[r] = 0u;
        }
        const uint32_t d = valid ? (key[r] >> shift) & 255u : 256u;  // 256: no key
        const unsigned peers = __match_any_sync(SS_FULL, d);
        const uint32_t cnt = valid ? wcnt[w][d] : 0u;
        rank[r] = cnt + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = cnt + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {  // per digit: exclusive prefix of the warps' counts, and the tile's total
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < RS_WARPS; ++k) {
            const uint32_t t = wcnt[k][d];
            wcnt[k][d] = run;
            run += t;
        }
        toff[d] = rs_block_excl(run, wtmp);  // first slot of digit d in the tile
    }
    __syncthreads();
    // place the tile in digit order
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & 255u;
            const uint32_t lp = toff[d] + wcnt[w][d] + rank[r];
            if (C == 1) {
                srec[lp] = make_uint2(key[r], aux[r]);
            } else {
                skey[lp] = key[r];
                sval[lp] = __ldg(reinterpret_cast<const float4 *>(vin) + i);
            }
        }
    }
    __syncthreads();
    // copy out in digit order: slot j of the tile goes to goff[d] + (j - toff[d])
    const int tn = (int)(n - tile0 < TILE ? n - tile0 : TILE);
    for (int j = threadIdx.x; j < tn; j += RS_THREADS) {
        if (C == 1) {
            const uint2 rec = srec[j];
            const uint32_t d = (rec.x >> shift) & 255u;
            reinterpret_cast<uint2 *>(kout)[(int64_t)goff[d] + (j - toff[d])] = rec;
        } else {
            const uint32_t k = skey[j];
            const uint32_t d = (k >> shift) & 255u;
            const int64_t pos = (int64_t)goff[d] + (j - toff[d]);
            kout[pos] = k;
            reinterpret_cast<float4 *>(vout)[pos] = sval[j];
        }
    }
}

template <int C>
static cudaError_t radix_sort_c(uint32_t *k_a, float *v_a, uint32_t *k_b, float *v_b, int64_t n,
                                int key_bits, uint32_t *hist, uint32_t *tmp, uint32_t **k_out,
                                float **v_out, cudaStream_t stream) {
    constexpr int TILE = RS_THREADS * RsCfg<C>::ROUNDS;
    const int64_t G = (n + TILE - 1) / TILE;
    if (G > 0x7fffffff) return cudaErrorInvalidValue;
    uint32_t *ki = k_a, *ko = k_b;
    float *vi = v_a, *vo = v_b;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_radix_hist<C><<<(unsigned)G, RS_THREADS, 0, stream>>>(ki, n, shift, hist, G);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // in place: each element is read before its slot is written (k_scan_tiles)
        e = launch_scan_u32(hist, hist, 256 * G, tmp, stream);
        if (e != cudaSuccess) return e;
        k_radix_scatter<C><<<(unsigned)G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, n, shift, hist, G);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t *kt = ki; ki = ko; ko = kt;
        float *vt = vi; vi = vo; vo = vt;
    }
    *k_out = ki;
    *v_out = vi;
    return cudaSuccess;
}

cudaError_t launch_radix_sort(uint32_t *k_a, float *v_a, uint32_t *k_b, float *v_b, int64_t n,
                              int channels, int key_bits, uint32_t *hist, uint32_t *tmp,
                              uint32_t **k_out, float **v_out, cudaStream_t stream) {
    *k_out = k_a;
    *v_out = v_a;
    if (n <= 1) return cudaSuccess;
    if (n > 0xffffffffll) return cudaErrorInvalidValue;  // 32-bit output offsets
    return channels == 4
               ? radix_sort_c<4>(k_a, v_a, k_b, v_b, n, key_bits, hist, tmp, k_out, v_out, stream)
               : radix_sort_c<1>(k_a, v_a, k_b, v_b, n, key_bits, hist, tmp, k_out, v_out, stream);
}

// ------------------------------------------------------------- run reduce
//
// Runs of equal keys in the sorted chunk are compacted first (head flags, a
// prefix sum, the heads' positions), so that consecutive threads own
// consecutive runs: thread t sums run t sequentially (Kahan) and adds it to
// acc[key] with a plain read-modify-write (one run per key per chunk, and
// chunks in stream order).  Every sum is taken in a fixed order.

template <int C>
__global__ void k_run_heads(const uint32_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || rs_key<C>(keys, i) != rs_key<C>(keys, i - 1)) ? 1u : 0u;
}

// starts[runidx[i]] = i at run heads; starts[R] = n (runidx[n] = R)
template <int C>
__global__ void k_run_starts(const uint32_t *__restrict__ keys, int64_t n,
                             const uint32_t *__restrict__ runidx, uint32_t *__restrict__ starts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        starts[runidx[n]] = (uint32_t)n;
        return;
    }
    if (i == 0 || rs_key<C>(keys, i) != rs_key<C>(keys, i - 1)) starts[runidx[i]] = (uint32_t)i;
}

template <int C>
__global__ void k_run_reduce(const uint32_t *__restrict__ keys, const float *__restrict__ vals,
                             const uint32_t *__restrict__ starts, const uint32_t *__restrict__ nruns,
                             float *__restrict__ acc) {
    const uint32_t R = *nruns;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < R; t += gridDim.x * blockDim.x) {
        const uint32_t j0 = __ldg(starts + t), j1 = __ldg(starts + t + 1);
        const uint32_t k = rs_key<C>(keys, j0);
        float s[C], c[C];
#pragma unroll
        for (int q = 0; q < C; ++q) { s[q] = 0.f; c[q] = 0.f; }
        for (uint32_t j = j0; j < j1; ++j) {
            float v[C];
            if (C == 4) {
                const float4 v4 = __ldg(reinterpret_cast<const float4 *>(vals) + j);
                v[0] = v4.x; v[1 % C] = v4.y; v[2 % C] = v4.z; v[3 % C] = v4.w;
            } else {
                v[0] = __uint_as_float(__ldg(reinterpret_cast<const uint2 *>(keys) + j).y);
            }
#pragma unroll
            for (int q = 0; q < C; ++q) {  // Kahan
                const float y = v[q] - c[q];
                const float tt = s[q] + y;
                c[q] = (tt - s[q]) - y;
                s[q] = tt;
            }
        }
#pragma unroll
        for (int q = 0; q < C; ++q) acc[(int64_t)k * C + q] += s[q];
    }
}

template <int C>
static cudaError_t seg_reduce_c(const uint32_t *keys, const float *vals, int64_t n, float *acc,
                                uint32_t *scratch, uint32_t *tmp, cudaStream_t stream) {
    uint32_t *flag = scratch;            // n + 1: head flags, then their prefix sums
    uint32_t *starts = scratch + n + 1;  // R + 1
    const int64_t blocks = (n + 1 + 255) / 256;
    k_run_heads<C><<<(unsigned)blocks, 256, 0, stream>>>(keys, n, flag);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan_u32(flag, flag, n, tmp, stream);  // flag[n] = number of runs
    if (e != cudaSuccess) return e;
    k_run_starts<C><<<(unsigned)blocks, 256, 0, stream>>>(keys, n, flag, starts);
    note_launch();
    k_run_reduce<C><<<(unsigned)(8 * device_sm_count()), 256, 0, stream>>>(keys, vals, starts,
                                                                          flag + n, acc);
    note_launch();
    return cudaGetLastError();
}

int64_t seg_reduce_scratch_elems(int64_t n) { return 2 * (n + 1); }

cudaError_t launch_seg_reduce(const uint32_t *keys, const float *vals, int64_t n, int channels,
                              float *acc, uint32_t *scratch, uint32_t *tmp, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    if (n >= 0xffffffffll || (n + 1 + 255) / 256 > 0x7fffffff) return cudaErrorInvalidValue;
    return channels == 4 ? seg_reduce_c<4>(keys, vals, n, acc, scratch, tmp, stream)
                         : seg_reduce_c<1>(keys, vals, n, acc, scratch, tmp, stream);
}

}  // namespace tp
