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
// One pass sorts by the 8-bit digit d = (key >> shift) & 255, stably:
//   1. k_radix_hist: per tile of RS_TILE keys, the digit histogram, stored
//      digit-major (hist[d * G + tile]);
//   2. exclusive scan of hist: the first output slot of (digit, tile);
//   3. k_radix_scatter: each warp ranks its 32-key rounds with
//      __match_any_sync (lanes with one digit, in lane order) on top of the
//      warp's running digit counts; warps own consecutive sub-tiles, so the
//      prefix of the warps' counts completes a stable rank within the tile.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                  // 32-key rounds per warp
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // 4096 keys per CTA

int64_t radix_hist_elems(int64_t n) { return 256 * ((n + RS_TILE - 1) / RS_TILE) + 1; }

__global__ void __launch_bounds__(RS_THREADS)
    k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist,
                 int64_t G) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&h[(__ldg(keys + i) >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * G + blockIdx.x] = h[threadIdx.x];
}

template <int C>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_scatter(const uint32_t *__restrict__ kin, const float *__restrict__ vin,
                    uint32_t *__restrict__ kout, float *__restrict__ vout, int64_t n, int shift,
                    const uint32_t *__restrict__ offs, int64_t G) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t goff[256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    goff[threadIdx.x] = __ldg(offs + (int64_t)threadIdx.x * G + blockIdx.x);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ROUNDS);
    uint32_t key[RS_ROUNDS], rank[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? __ldg(kin + i) : 0u;
        const uint32_t d = valid ? (key[r] >> shift) & 255u : 256u;  // 256: no key
        const unsigned peers = __match_any_sync(SS_FULL, d);
        const uint32_t cnt = valid ? wcnt[w][d] : 0u;
        rank[r] = cnt + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = cnt + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {  // exclusive prefix of the warps' counts, per digit
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < RS_WARPS; ++k) {
            const uint32_t t = wcnt[k][d];
            wcnt[k][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & 255u;
            const int64_t pos = (int64_t)goff[d] + wcnt[w][d] + rank[r];
            kout[pos] = key[r];
            if (C == 4)
                reinterpret_cast<float4 *>(vout)[pos] = __ldg(reinterpret_cast<const float4 *>(vin) + i);
            else
                vout[pos] = __ldg(vin + i);
        }
    }
}

cudaError_t launch_radix_sort(uint32_t *k_a, float *v_a, uint32_t *k_b, float *v_b, int64_t n,
                              int channels, int key_bits, uint32_t *hist, uint32_t *tmp,
                              uint32_t **k_out, float **v_out, cudaStream_t stream) {
    *k_out = k_a;
    *v_out = v_a;
    if (n <= 1) return cudaSuccess;
    if (n > 0xffffffffll) return cudaErrorInvalidValue;  // 32-bit output offsets
    const int64_t G = (n + RS_TILE - 1) / RS_TILE;
    if (G > 0x7fffffff) return cudaErrorInvalidValue;
    uint32_t *ki = k_a, *ko = k_b;
    float *vi = v_a, *vo = v_b;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_radix_hist<<<(unsigned)G, RS_THREADS, 0, stream>>>(ki, n, shift, hist, G);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // in place: each element is read before its slot is written (k_scan_tiles)
        e = launch_scan_u32(hist, hist, 256 * G, tmp, stream);
        if (e != cudaSuccess) return e;
        if (channels == 4)
            k_radix_scatter<4><<<(unsigned)G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, n, shift, hist, G);
        else
            k_radix_scatter<1><<<(unsigned)G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, n, shift, hist, G);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t *kt = ki; ki = ko; ko = kt;
        float *vt = vi; vi = vo; vo = vt;
    }
    *k_out = ki;
    *v_out = vi;
    return cudaSuccess;
}

// ------------------------------------------------------------- run reduce

template <int C>
__global__ void k_seg_reduce(const uint32_t *__restrict__ keys, const float *__restrict__ vals,
                             int64_t n, float *__restrict__ acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = __ldg(keys + i);
    if (i > 0 && __ldg(keys + i - 1) == k) return;  // not the first of its run
    float s[C], c[C];
#pragma unroll
    for (int q = 0; q < C; ++q) { s[q] = 0.f; c[q] = 0.f; }
    for (int64_t j = i; j < n && __ldg(keys + j) == k; ++j) {
        float v[C];
        if (C == 4) {
            const float4 v4 = __ldg(reinterpret_cast<const float4 *>(vals) + j);
            v[0] = v4.x; v[1 % C] = v4.y; v[2 % C] = v4.z; v[3 % C] = v4.w;
        } else {
            v[0] = __ldg(vals + j);
        }
#pragma unroll
        for (int q = 0; q < C; ++q) {  // Kahan
            const float y = v[q] - c[q];
            const float t = s[q] + y;
            c[q] = (t - s[q]) - y;
            s[q] = t;
        }
    }
    // one run per key in a chunk: a plain read-modify-write, in chunk order
#pragma unroll
    for (int q = 0; q < C; ++q) acc[(int64_t)k * C + q] += s[q];
}

cudaError_t launch_seg_reduce(const uint32_t *keys, const float *vals, int64_t n, int channels,
                              float *acc, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (channels == 4)
        k_seg_reduce<4><<<(unsigned)blocks, 256, 0, stream>>>(keys, vals, n, acc);
    else
        k_seg_reduce<1><<<(unsigned)blocks, 256, 0, stream>>>(keys, vals, n, acc);
    return cudaGetLastError();
}

}  // namespace tp
