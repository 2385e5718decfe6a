// api.cu -- the extern "C" boundary declared in include/tetproj.h.
//
// Host-side glue only: argument checks, ownership of device memory, the
// user-order <-> Hilbert-order permutations around each walk, and launch
// configuration.  Every step of the projection itself runs in kernels.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/tetproj.h"
#include "kernels.cuh"
#include "mesh_build.h"
#include "rstar.h"

using namespace tp;

// Segment plan of the sort-and-reduce backprojection for one (geometry, tile
// shape, ordering): per-ray segment counts and offsets, and the split of the
// tile blocks into chunks whose segments fit the sort buffers.  It depends on
// the mesh and the rays only, so it is built once and reused.
struct SegPlan {
    bool valid = false;
    uint64_t geo_uid = 0;
    int32_t tu = 0, tv = 0, morton = 0, channels = 0;
    int64_t nrays = 0, nblocks = 0;
    int32_t *count = nullptr;    // [nrays] segments per ray
    int32_t *ray_off = nullptr;  // [nrays] offset inside the ray's tile block
    int64_t *block_cnt = nullptr, *block_off = nullptr, *scan_tmp = nullptr;
    DevCounters *counters = nullptr;  // the counting walk's own counters
    std::vector<int64_t> chunk_b, chunk_s;  // chunk boundaries: blocks, segments
    int64_t max_chunk = 0;
    int64_t bytes = 0;
};

// Sort buffers (double-buffered keys and C-float values) and radix scratch.
struct SortWs {
    uint32_t *k[2] = {nullptr, nullptr};
    float *v[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr, *tmp = nullptr;
    int64_t cap = 0;
    int32_t cap_c = 0;
    int64_t bytes = 0;
};

// Segments per sort chunk: 2^29 at C = 1 (8-byte records, double-buffered:
// 8.6 GB), 2^27 at C = 4 (24 bytes per record: 6.4 GB).  Fewer chunks mean
// fewer walk/resume launch tails.
static int64_t seg_chunk(int channels) { return int64_t(1) << (channels == 4 ? 27 : 29); }

struct tetproj_mesh {
    int device = 0;
    TetRec32 *rec32 = nullptr;
    TetRec64 *rec64 = nullptr;
    BvhNode *bvh = nullptr;
    BFace32 *bfaces = nullptr;
    int32_t *perm = nullptr;
    int4 *vid = nullptr;
    RStarNode *rstar = nullptr;  // built on first use of TETPROJ_FLAG_RSTAR_ENTRY
    int64_t rstar_bytes = 0;
    DevCounters *counters = nullptr;
    int64_t nt = 0, nv = 0, nb = 0, nnodes = 0, nflipped = 0;
    int32_t root = 0;
    float radius = 0.f;
    double bbox[6] = {0, 0, 0, 0, 0, 0};
    // workspace per [precision][channels==4]: tet-ordered operand / accumulator
    void *ws[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t ws_bytes[2][2] = {{0, 0}, {0, 0}};
    // deferral queue of the filtered walk (see kernels.cu), and a second one
    // with an auxiliary stream so that resume kernels overlap the next chunk
    QEntry *q = nullptr;
    unsigned long long *q_count = nullptr;
    int64_t q_cap = 0;
    ResumeOverlap ov = {};
    bool ov_ready = false;
    // candidate entry faces per pixel of a launch chunk's angles (cone rays)
    int32_t *emap = nullptr;
    int64_t emap_cap = 0;
    int64_t base_bytes = 0;
    SegPlan plan;
    SortWs sort;
};

// Largest deferral queue (entries of 64 B); launches over more rays are chunked.
// Single-problem calls: 2^24 rays per chunk (queue and fix list 1.25 GB; two
// of them when a call has several chunks); on the 94M-ray jittered 96^3 step
// 1% faster than 2^23 (272.7 vs 275.5 ms), 2^22 was 2% slower.  A batch holds
// one queue pair for all its problems and runs rounds of 2^25 rays (2.5 GB
// each): on 24 jittered Kuhn meshes of 16^3-118^3 cells (1.6G rays, C = 4)
// 2,606 ms per forward + backprojection against 2,722 at 2^23.
static const int64_t kQueueMax = int64_t(1) << 24;
static const int64_t kBatchQueueMax = int64_t(1) << 25;

static std::atomic<uint64_t> g_geometry_uid{1};

struct tetproj_geometry {
    int device = 0;
    uint64_t uid = 0;  // distinguishes geometries for cached segment plans
    AngleFrame *frames = nullptr;
    int32_t nu = 0, nv = 0, na = 0;
    double du = 0, dv = 0, dso = 0, dsd = 0;
};

static tetproj_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return TETPROJ_OK;
    if (e == cudaErrorMemoryAllocation) return TETPROJ_ERR_OOM;
    return TETPROJ_ERR_CUDA;
}
#define TP_CUDA(x)                                         \
    do {                                                   \
        cudaError_t _e = (x);                              \
        if (_e != cudaSuccess) return cuda_status(_e);     \
    } while (0)

template <typename T>
static cudaError_t dalloc(T **p, int64_t n, int64_t &bytes) {
    cudaError_t e = cudaMalloc((void **)p, (size_t)(n > 0 ? n : 1) * sizeof(T));
    if (e == cudaSuccess) bytes += (n > 0 ? n : 1) * (int64_t)sizeof(T);
    return e;
}

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

extern "C" {

int32_t tetproj_version(void) { return 201; }

int64_t tetproj_launch_count(void) { return (int64_t)launch_count(); }

void tetproj_default_options(tetproj_options *o) {
    if (!o) return;
    o->precision = TETPROJ_FILTERED;
    o->channels = 1;
    o->tile_u = 16;
    o->tile_v = 8;
    o->order = TETPROJ_ORDER_MORTON;
    o->scatter = TETPROJ_SCATTER_ATOMIC;
    o->max_steps = 0;
    o->flags = 0;
}

const char *tetproj_status_string(tetproj_status s) {
    switch (s) {
        case TETPROJ_OK: return "ok";
        case TETPROJ_ERR_ARG: return "invalid argument";
        case TETPROJ_ERR_INDEX: return "vertex index out of range or repeated in a tet";
        case TETPROJ_ERR_DEGENERATE_TET: return "zero-volume tet";
        case TETPROJ_ERR_NONMANIFOLD: return "non-manifold mesh (face shared by >2 tets or overlapping tets)";
        case TETPROJ_ERR_NONCONVEX: return "mesh boundary is not convex (or mesh not connected)";
        case TETPROJ_ERR_CUDA: return "CUDA runtime error";
        case TETPROJ_ERR_OOM: return "out of memory";
        case TETPROJ_ERR_RAY_LIMIT: return "a ray walk exceeded max_steps or met an inconsistent tet";
        case TETPROJ_ERR_TIMEOUT: return "a bounded device wait timed out";
        case TETPROJ_ERR_SOURCE_INSIDE: return "a ray source lies inside the mesh";
        case TETPROJ_ERR_TOO_LARGE: return "size exceeds a documented limit";
        default: return "unknown status";
    }
}

static void plan_free(SegPlan &pl) {
    cudaFree(pl.count);
    cudaFree(pl.ray_off);
    cudaFree(pl.block_cnt);
    cudaFree(pl.block_off);
    cudaFree(pl.scan_tmp);
    cudaFree(pl.counters);
    pl = SegPlan();
}

static void sort_free(SortWs &w) {
    for (int i = 0; i < 2; ++i) {
        cudaFree(w.k[i]);
        cudaFree(w.v[i]);
    }
    cudaFree(w.hist);
    cudaFree(w.tmp);
    w = SortWs();
}

// releases whatever part of `o` exists (also after a failed overlap_create)
static void overlap_release(ResumeOverlap &o) {
    cudaFree(o.q2);
    cudaFree(o.q2_count);
    if (o.aux) cudaStreamDestroy(o.aux);
    for (int j = 0; j < 2; ++j) {
        if (o.ev_fast[j]) cudaEventDestroy(o.ev_fast[j]);
        if (o.ev_res[j]) cudaEventDestroy(o.ev_res[j]);
    }
    if (o.ev_start) cudaEventDestroy(o.ev_start);
    o = ResumeOverlap{};
}

// second queue of `cap` entries, the auxiliary stream (highest priority, so
// that a chunk's resume is not starved by the next chunk's walk) and events
static cudaError_t overlap_create(ResumeOverlap &o, int64_t cap) {
    o = ResumeOverlap{};
    int lo = 0, hi = 0;
    cudaError_t e = cudaMalloc((void **)&o.q2, (size_t)queue_bytes(cap));
    if (e == cudaSuccess) e = cudaMalloc((void **)&o.q2_count, kQueueCountBytes);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&o.aux, cudaStreamNonBlocking, hi);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
        e = cudaEventCreateWithFlags(&o.ev_fast[j], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o.ev_res[j], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o.ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) overlap_release(o);
    return e;
}

static void overlap_free(tetproj_mesh *m) {
    if (!m->ov_ready) return;
    overlap_release(m->ov);
    m->ov_ready = false;
}

static void mesh_free(tetproj_mesh *m) {
    if (!m) return;
    overlap_free(m);
    plan_free(m->plan);
    sort_free(m->sort);
    cudaFree(m->rec32);
    cudaFree(m->rec64);
    cudaFree(m->bvh);
    cudaFree(m->bfaces);
    cudaFree(m->perm);
    cudaFree(m->vid);
    cudaFree(m->rstar);
    cudaFree(m->counters);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) cudaFree(m->ws[i][j]);
    cudaFree(m->q);
    cudaFree(m->q_count);
    cudaFree(m->emap);
    delete m;
}

tetproj_status tetproj_mesh_create(const double *vertices, int64_t nv, const int32_t *tets,
                                   int64_t nt, tetproj_mesh **out) {
    if (!out) return TETPROJ_ERR_ARG;
    *out = nullptr;
    HostMesh H;
    tetproj_status st;
    try {
        st = build_host_mesh(vertices, nv, tets, nt, H);
    } catch (const std::bad_alloc &) {
        return TETPROJ_ERR_OOM;
    }
    if (st != TETPROJ_OK) return st;
    tetproj_mesh *m = new (std::nothrow) tetproj_mesh();
    if (!m) return TETPROJ_ERR_OOM;
    cudaGetDevice(&m->device);
    m->nt = H.nt;
    m->nv = H.nv;
    m->nb = H.nb;
    m->nnodes = (int64_t)H.bvh.size();
    m->nflipped = H.nflipped;
    m->root = H.root;
    m->radius = H.radius;
    std::memcpy(m->bbox, H.bbox, sizeof(m->bbox));
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = upload(&m->rec32, H.rec32);
    if (e == cudaSuccess) e = upload(&m->rec64, H.rec64);
    if (e == cudaSuccess) e = upload(&m->bvh, H.bvh);
    if (e == cudaSuccess) e = upload(&m->bfaces, H.bfaces);
    if (e == cudaSuccess) e = upload(&m->perm, H.perm);
    if (e == cudaSuccess) e = upload(&m->vid, H.vid);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->counters, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMemset(m->counters, 0, sizeof(DevCounters));
    if (e != cudaSuccess) {
        mesh_free(m);
        return cuda_status(e);
    }
    m->base_bytes = (int64_t)(H.rec32.size() * sizeof(TetRec32) + H.rec64.size() * sizeof(TetRec64) +
                              H.bvh.size() * sizeof(BvhNode) + H.bfaces.size() * sizeof(BFace32) +
                              H.perm.size() * sizeof(int32_t) + H.vid.size() * sizeof(int4) +
                              sizeof(DevCounters));
    *out = m;
    return TETPROJ_OK;
}

tetproj_status tetproj_mesh_destroy(tetproj_mesh *m) {
    if (!m) return TETPROJ_ERR_ARG;
    cudaDeviceSynchronize();
    mesh_free(m);
    return TETPROJ_OK;
}

tetproj_status tetproj_mesh_get_info(const tetproj_mesh *m, tetproj_mesh_info *o) {
    if (!m || !o) return TETPROJ_ERR_ARG;
    o->nt = m->nt;
    o->nv = m->nv;
    o->nboundary = m->nb;
    o->nbvh_nodes = m->nnodes;
    o->nflipped = m->nflipped;
    int64_t b = m->base_bytes + queue_bytes(m->q_cap) * (m->ov_ready ? 2 : 1) +
                (m->q_count ? (int64_t)kQueueCountBytes : 0) + m->emap_cap * (int64_t)sizeof(int32_t) +
                m->plan.bytes + m->sort.bytes + m->rstar_bytes;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) b += m->ws_bytes[i][j];
    o->device_bytes = b;
    std::memcpy(o->bbox, m->bbox, sizeof(o->bbox));
    return TETPROJ_OK;
}

static tetproj_status ensure_ws(tetproj_mesh *m, int precision, int channels) {
    int pi = precision == TETPROJ_PLAIN_FP64 ? 1 : 0, ci = channels == 4 ? 1 : 0;
    if (m->ws[pi][ci]) return TETPROJ_OK;
    int64_t bytes = m->nt * channels * (pi ? 8 : 4);
    void *p = nullptr;
    TP_CUDA(cudaMalloc(&p, (size_t)bytes));
    m->ws[pi][ci] = p;
    m->ws_bytes[pi][ci] = bytes;
    return TETPROJ_OK;
}

// True while `s` is being captured into a CUDA graph: no allocation then (a
// query that fails counts as capturing).
static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Deferral queue able to hold one launch chunk of up to min(nrays, kQueueMax)
// rays; with allow_ov, also the overlap resources when there are several chunks.
static tetproj_status ensure_queue(tetproj_mesh *m, int64_t nrays, bool allow_ov) {
    int64_t need = nrays < kQueueMax ? nrays : kQueueMax;
    need = ((need + 4095) / 4096) * 4096;
    // the second queue and the auxiliary stream only pay off with several chunks
    const bool want_ov = allow_ov && nrays > kQueueMax;
    if (m->q_cap >= need && m->q_count && (!want_ov || m->ov_ready)) return TETPROJ_OK;
    if (m->q_cap < need || !m->q_count) {
        cudaDeviceSynchronize();  // the queues may be in use by earlier calls
        overlap_free(m);
        cudaFree(m->q);
        m->q = nullptr;
        m->q_cap = 0;
        TP_CUDA(cudaMalloc((void **)&m->q, (size_t)queue_bytes(need)));
        if (!m->q_count) TP_CUDA(cudaMalloc((void **)&m->q_count, kQueueCountBytes));
        m->q_cap = need;
    }
    if (want_ov && !m->ov_ready) {
        TP_CUDA(overlap_create(m->ov, m->q_cap));
        m->ov_ready = true;
    }
    return TETPROJ_OK;
}

// the overlap resources when this mesh has them (calls of several chunks)
static const ResumeOverlap *overlap_of(const tetproj_mesh *m) {
    return m->ov_ready ? &m->ov : nullptr;
}

tetproj_status tetproj_mesh_reserve(tetproj_mesh *m, int32_t precision, int32_t channels) {
    if (!m || (precision != TETPROJ_FILTERED && precision != TETPROJ_PLAIN_FP64) ||
        (channels != 1 && channels != 4))
        return TETPROJ_ERR_ARG;
    tetproj_status st = ensure_ws(m, precision, channels);
    if (st == TETPROJ_OK && precision == TETPROJ_FILTERED) st = ensure_queue(m, kQueueMax, false);
    // the FP64 accumulator the filtered backprojection uses by default at C = 1,
    // and at C = 4 on meshes small enough to be dense (two-level accumulation)
    if (st == TETPROJ_OK && precision == TETPROJ_FILTERED &&
        (channels == 1 || m->nt * channels <= (int64_t(1) << 20)))
        st = ensure_ws(m, TETPROJ_PLAIN_FP64, channels);
    return st;
}

tetproj_status tetproj_mesh_topology_host(const double *V, int64_t nv, const int32_t *T,
                                          int64_t nt, int32_t *adj_out, int64_t *nboundary,
                                          int64_t *nflipped) {
    try {
        return topology_host(V, nv, T, nt, adj_out, nboundary, nflipped);
    } catch (const std::bad_alloc &) {
        return TETPROJ_ERR_OOM;
    }
}

tetproj_status tetproj_mesh_stats_reset(tetproj_mesh *m, void *stream) {
    if (!m) return TETPROJ_ERR_ARG;
    TP_CUDA(cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), (cudaStream_t)stream));
    return TETPROJ_OK;
}

tetproj_status tetproj_mesh_stats_read(tetproj_mesh *m, void *stream, tetproj_stats *o) {
    if (!m || !o) return TETPROJ_ERR_ARG;
    DevCounters c;
    TP_CUDA(cudaMemcpyAsync(&c, m->counters, sizeof(c), cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream));
    TP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    o->rays = (int64_t)c.rays;
    o->hits = (int64_t)c.hits;
    o->segments = (int64_t)c.segments;
    o->fp64_filter = (int64_t)c.fp64;
    o->exact = (int64_t)c.exact;
    o->sos = (int64_t)c.sos;
    o->bvh_nodes = (int64_t)c.bvh_nodes;
    o->bvh_faces = (int64_t)c.bvh_faces;
    o->deferred = (int64_t)c.deferred;
    o->error = c.error;
    o->error_count = c.error_count;
    o->grazing = (int64_t)c.grazing;
    return TETPROJ_OK;
}

tetproj_status tetproj_geometry_create(double dso, double dsd, int32_t nu, int32_t nv, double du,
                                       double dv, const double *angles, int32_t nangles,
                                       tetproj_geometry **out) {
    if (!out) return TETPROJ_ERR_ARG;
    *out = nullptr;
    if (!angles || nu < 1 || nv < 1 || nangles < 1 || !(dso > 0) || !(dsd > dso) || !(du > 0) ||
        !(dv > 0))
        return TETPROJ_ERR_ARG;
    if ((int64_t)nu * nv * nangles >= (int64_t(1) << 40)) return TETPROJ_ERR_TOO_LARGE;
    std::vector<AngleFrame> F(nangles);
    for (int a = 0; a < nangles; ++a) {
        double c = std::cos(angles[a]), s = std::sin(angles[a]);
        AngleFrame &f = F[a];
        f.S[0] = dso * c;
        f.S[1] = dso * s;
        f.S[2] = 0.0;
        f.C[0] = f.S[0] - dsd * c;
        f.C[1] = f.S[1] - dsd * s;
        f.C[2] = 0.0;
        f.U[0] = -s;
        f.U[1] = c;
        f.U[2] = 0.0;
        f.V[0] = 0.0;
        f.V[1] = 0.0;
        f.V[2] = 1.0;
    }
    tetproj_geometry *g = new (std::nothrow) tetproj_geometry();
    if (!g) return TETPROJ_ERR_OOM;
    cudaGetDevice(&g->device);
    g->nu = nu;
    g->nv = nv;
    g->na = nangles;
    g->du = du;
    g->dv = dv;
    g->dso = dso;
    g->dsd = dsd;
    g->uid = g_geometry_uid.fetch_add(1);
    cudaError_t e = upload(&g->frames, F);
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e);
    }
    *out = g;
    return TETPROJ_OK;
}

tetproj_status tetproj_geometry_destroy(tetproj_geometry *g) {
    if (!g) return TETPROJ_ERR_ARG;
    cudaDeviceSynchronize();
    cudaFree(g->frames);
    delete g;
    return TETPROJ_OK;
}

static GeoView geo_view(const tetproj_geometry *g) {
    GeoView v;
    v.frames = g->frames;
    v.nu = g->nu;
    v.nv = g->nv;
    v.na = g->na;
    v.du = g->du;
    v.dv = g->dv;
    return v;
}

tetproj_status tetproj_geometry_rays(const tetproj_geometry *g, const int64_t *idx, int64_t n,
                                     double *src, double *dst, void *stream) {
    if (!g || n < 0 || (n > 0 && (!src || !dst))) return TETPROJ_ERR_ARG;
    TP_CUDA(launch_geometry_rays(geo_view(g), idx, n, src, dst, (cudaStream_t)stream));
    return TETPROJ_OK;
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static tetproj_status check_opts(const tetproj_options *in, tetproj_options &o) {
    if (in) o = *in;
    else tetproj_default_options(&o);
    if (o.precision != TETPROJ_FILTERED && o.precision != TETPROJ_PLAIN_FP64) return TETPROJ_ERR_ARG;
    if (o.channels != 1 && o.channels != 4) return TETPROJ_ERR_ARG;
    auto pow2 = [](int v) { return v >= 1 && v <= 32 && (v & (v - 1)) == 0; };
    if (!pow2(o.tile_u) || !pow2(o.tile_v)) return TETPROJ_ERR_ARG;
    int t = o.tile_u * o.tile_v;
    if (t < 32 || t > 256) return TETPROJ_ERR_ARG;
    if (o.order != TETPROJ_ORDER_ROW && o.order != TETPROJ_ORDER_MORTON) return TETPROJ_ERR_ARG;
    if (o.scatter != TETPROJ_SCATTER_ATOMIC && o.scatter != TETPROJ_SCATTER_WARP &&
        o.scatter != TETPROJ_SCATTER_SORT)
        return TETPROJ_ERR_ARG;
    if (o.max_steps < 0 ||
        (o.flags & ~(TETPROJ_FLAG_RSTAR_ENTRY | TETPROJ_FLAG_ACC64 | TETPROJ_FLAG_ACC32)) != 0 ||
        ((o.flags & TETPROJ_FLAG_ACC64) && (o.flags & TETPROJ_FLAG_ACC32)))
        return TETPROJ_ERR_ARG;
    return TETPROJ_OK;
}

static KParams base_params(const tetproj_mesh *m, const tetproj_options &o) {
    KParams p;
    std::memset(&p, 0, sizeof(p));
    p.m.rec32 = m->rec32;
    p.m.rec64 = m->rec64;
    p.m.vid = m->vid;
    p.m.bvh = m->bvh;
    p.m.bfaces = m->bfaces;
    p.m.perm = m->perm;
    p.m.nt = m->nt;
    p.m.nb = m->nb;
    p.m.nnodes = m->nnodes;
    p.m.root = m->root;
    p.m.radius = m->radius;
    p.m.counters = m->counters;
    p.tu = o.tile_u;
    p.tv = o.tile_v;
    p.log_tu = ilog2(o.tile_u);
    p.log_tv = ilog2(o.tile_v);
    p.morton = o.order == TETPROJ_ORDER_MORTON;
    p.scatter = o.scatter;
    int64_t cb = (int64_t)std::ceil(std::cbrt((double)m->nt));
    int64_t def = 64 + 16 * cb;
    int64_t ms = o.max_steps > 0 ? o.max_steps : def;
    if (ms > m->nt + 1) ms = m->nt + 1;
    p.max_steps = (int32_t)ms;
    p.smem_nodes = (int32_t)(m->nnodes < 64 ? m->nnodes : 64);
    p.entry = (o.flags & TETPROJ_FLAG_RSTAR_ENTRY) ? ENTRY_RSTAR : ENTRY_BVH;
    p.m.rstar = m->rstar;
    return p;
}

// The R*-tree of the boundary faces, built on the host from the device copy of
// the faces on first use (synchronous).
static tetproj_status ensure_rstar(tetproj_mesh *m, KParams &p) {
    if (!m->rstar) {
        std::vector<BFace32> faces((size_t)m->nb);
        TP_CUDA(cudaMemcpy(faces.data(), m->bfaces, sizeof(BFace32) * m->nb,
                           cudaMemcpyDeviceToHost));
        std::vector<RStarNode> nodes;
        rstar_build(faces, nodes);
        if (rstar_check(faces, nodes).depth > RSTAR_MAX_DEPTH) return TETPROJ_ERR_TOO_LARGE;
        cudaError_t e = upload(&m->rstar, nodes);
        if (e != cudaSuccess) return cuda_status(e);
        m->rstar_bytes = (int64_t)(nodes.size() * sizeof(RStarNode));
    }
    p.m.rstar = m->rstar;
    return TETPROJ_OK;
}

// Calls without an R*-tree variant reject the flag.
static bool rstar_unsupported(const tetproj_options &o) {
    return (o.flags & TETPROJ_FLAG_RSTAR_ENTRY) != 0;
}

static void set_cone(KParams &p, const tetproj_geometry *g) {
    p.src_kind = 0;
    p.g = geo_view(g);
    p.tiles_u = (g->nu + p.tu - 1) / p.tu;
    p.tiles_v = (g->nv + p.tv - 1) / p.tv;
    p.nrays = (int64_t)g->na * g->nu * g->nv;
}

static tetproj_status attach_queue(tetproj_mesh *m, KParams &p, const tetproj_options &o,
                                   cudaStream_t s) {
    if (o.precision != TETPROJ_FILTERED) return TETPROJ_OK;
    // under graph capture a call without the overlap resources runs its
    // chunks on one stream instead of allocating them
    tetproj_status st = ensure_queue(m, p.nrays, !capturing(s));
    if (st != TETPROJ_OK) return st;
    p.q = m->q;
    p.q_count = m->q_count;
    p.q_cap = m->q_cap;
    return TETPROJ_OK;
}

// The entry map of the fast walk (KParams::emap): for filtered cone-beam
// calls with the BVH entry whose source circle lies outside the mesh's
// bounding sphere, a buffer for the angles one launch chunk touches.  Only a
// hint (the walk verifies every candidate), so it is left out under graph
// capture when not yet allocated, or when it would exceed 256 MB.
static tetproj_status attach_emap(tetproj_mesh *m, KParams &p, const tetproj_options &o,
                                  const tetproj_geometry *geo, cudaStream_t s) {
    p.emap_buf = nullptr;
    p.emap_cap = 0;
    if (o.precision != TETPROJ_FILTERED || p.entry != ENTRY_BVH || p.src_kind != 0 || !geo ||
        !(geo->dso > 1.75 * (double)m->radius) || p.q_cap <= 0)
        return TETPROJ_OK;
    const int64_t pix = (int64_t)geo->nu * geo->nv;
    const int64_t need = (p.q_cap / pix + 2) * pix;
    if (need > (int64_t(1) << 26)) return TETPROJ_OK;
    if (m->emap_cap < need) {
        if (capturing(s)) return TETPROJ_OK;
        cudaDeviceSynchronize();  // an earlier call may still read the old map
        cudaFree(m->emap);
        m->emap = nullptr;
        m->emap_cap = 0;
        TP_CUDA(cudaMalloc((void **)&m->emap, (size_t)need * sizeof(int32_t)));
        m->emap_cap = need;
    }
    p.emap_buf = m->emap;
    p.emap_cap = m->emap_cap;
    return TETPROJ_OK;
}

static tetproj_status run_forward(tetproj_mesh *m, KParams &p, const tetproj_options &o,
                                  const void *mu, void *out, cudaStream_t s,
                                  const tetproj_geometry *geo = nullptr) {
    if (p.entry == ENTRY_RSTAR) {  // the paper's entry structure: filtered path, C = 1
        if (o.precision != TETPROJ_FILTERED || o.channels != 1) return TETPROJ_ERR_ARG;
        tetproj_status st = ensure_rstar(m, p);
        if (st != TETPROJ_OK) return st;
    }
    tetproj_status st = ensure_ws(m, o.precision, o.channels);
    if (st == TETPROJ_OK) st = attach_queue(m, p, o, s);
    if (st == TETPROJ_OK) st = attach_emap(m, p, o, geo, s);
    if (st != TETPROJ_OK) return st;
    void *ws = m->ws[o.precision == TETPROJ_PLAIN_FP64][o.channels == 4];
    int f64 = o.precision == TETPROJ_PLAIN_FP64;
    TP_CUDA(launch_gather_perm(m->perm, m->nt, o.channels, f64, mu, ws, s));
    p.in = ws;
    p.out = out;
    TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_FWD, s, overlap_of(m)));
    return TETPROJ_OK;
}

// Accumulator of the filtered backprojection with atomic or warp-aggregated
// scatter: FP64 unless TETPROJ_FLAG_ACC32, or C = 4 without TETPROJ_FLAG_ACC64 (measured on GB300:
// at C = 1 the FP64 reduction is also the faster one; at C = 4 it needs four
// 8-byte reductions per segment against one 16-byte FP32 one).
static bool use_acc64(const tetproj_options &o) {
    if (o.precision != TETPROJ_FILTERED || o.scatter == TETPROJ_SCATTER_SORT) return false;
    if (o.flags & TETPROJ_FLAG_ACC64) return true;
    if (o.flags & TETPROJ_FLAG_ACC32) return false;
    return o.channels == 1;
}

// Dense problems (few tets, many rays) at C = 4: a tet collects up to ~10^5
// FP32 reductions per call, and their rounding drifts toward 1e-5 relative.
// There the default FP32 accumulation is two-level: the walk's FP32
// accumulator is moved into an FP64 one after every chunk of at most
// dense_chunk_rays rays, so no FP32 sum holds more than a few thousand terms
// (FP64 reductions instead cost 1.7-2.6x at C = 4, four 8-byte reductions per
// segment).  Dense: nt C <= 2^20 elements and >= 64 rays per element.
static bool dense_acc(int64_t nt, int channels, int64_t nrays) {
    const int64_t n = nt * channels;
    return n <= (int64_t(1) << 20) && nrays >= 64 * n;
}
// Rays per merge interval: about 8192 FP32 reductions per tet, estimating a
// ray's segments through a compact mesh of nt tets as 1.5 (nt / 6)^(1/3) + 1
// (a cube of n^3 cells has 6 n^3 tets); at least 2^18 rays.
static int64_t dense_chunk_rays(int64_t nt) {
    const double spr = 1.5 * std::cbrt((double)nt / 6.0) + 1.0;
    const double c = 8192.0 * (double)nt / spr;
    return c < (double)(int64_t(1) << 18) ? (int64_t(1) << 18)
                                          : (c > 1e15 ? (int64_t)1e15 : (int64_t)c);
}

static tetproj_status run_backward(tetproj_mesh *m, KParams &p, const tetproj_options &o,
                                   const void *y, void *mu_out, cudaStream_t s,
                                   const tetproj_geometry *geo = nullptr) {
    if (rstar_unsupported(o)) return TETPROJ_ERR_ARG;
    if ((o.flags & TETPROJ_FLAG_ACC64) && o.precision == TETPROJ_FILTERED &&
        o.scatter == TETPROJ_SCATTER_SORT)
        return TETPROJ_ERR_ARG;  // FP64 accumulation is an atomic-scatter variant
    if (use_acc64(o)) {
        // FP32 walk, FP64 accumulator (the plain path's workspace), one rounding at the end
        tetproj_status st = ensure_ws(m, TETPROJ_PLAIN_FP64, o.channels);
        if (st == TETPROJ_OK) st = attach_queue(m, p, o, s);
        if (st == TETPROJ_OK) st = attach_emap(m, p, o, geo, s);
        if (st != TETPROJ_OK) return st;
        void *ws = m->ws[1][o.channels == 4];
        TP_CUDA(cudaMemsetAsync(ws, 0, (size_t)m->ws_bytes[1][o.channels == 4], s));
        p.in = y;
        p.out = ws;
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD64, s, overlap_of(m)));
        TP_CUDA(launch_scatter_perm_d2f(m->perm, m->nt, o.channels,
                                        reinterpret_cast<const double *>(ws),
                                        reinterpret_cast<float *>(mu_out), s));
        return TETPROJ_OK;
    }
    tetproj_status st = ensure_ws(m, o.precision, o.channels);
    if (st == TETPROJ_OK) st = attach_queue(m, p, o, s);
    if (st == TETPROJ_OK) st = attach_emap(m, p, o, geo, s);
    if (st != TETPROJ_OK) return st;
    void *ws = m->ws[o.precision == TETPROJ_PLAIN_FP64][o.channels == 4];
    int f64 = o.precision == TETPROJ_PLAIN_FP64;
    TP_CUDA(cudaMemsetAsync(ws, 0, (size_t)m->ws_bytes[f64][o.channels == 4], s));
    p.in = y;
    p.out = ws;
    if (!f64 && !(o.flags & TETPROJ_FLAG_ACC32) && dense_acc(m->nt, o.channels, p.nrays)) {
        st = ensure_ws(m, TETPROJ_PLAIN_FP64, o.channels);
        if (st != TETPROJ_OK) return st;
        void *ws64 = m->ws[1][o.channels == 4];
        TP_CUDA(cudaMemsetAsync(ws64, 0, (size_t)m->ws_bytes[1][o.channels == 4], s));
        AccMerge mg{reinterpret_cast<float *>(ws), reinterpret_cast<double *>(ws64),
                    m->nt * o.channels, dense_chunk_rays(m->nt)};
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD, s, overlap_of(m), &mg));
        TP_CUDA(launch_scatter_perm_d2f(m->perm, m->nt, o.channels,
                                        reinterpret_cast<const double *>(ws64),
                                        reinterpret_cast<float *>(mu_out), s));
        return TETPROJ_OK;
    }
    TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD, s, overlap_of(m)));
    TP_CUDA(launch_scatter_perm(m->perm, m->nt, o.channels, f64, ws, mu_out, s));
    return TETPROJ_OK;
}

// ------------------------------------------ sort-and-reduce backprojection

// Builds (or reuses) the segment plan of (mesh, geometry, tile options):
// a counting walk (trace mode, no tets stored) gives each ray's number of
// segments; per tile block their exclusive prefix (ray_off) and total; a scan
// of the totals gives each block's first segment.  Chunks of consecutive
// blocks hold at most kSegChunk segments and q_cap rays.  Synchronous.
static tetproj_status ensure_plan(tetproj_mesh *m, const tetproj_geometry *geo, const KParams &p,
                                  int channels, cudaStream_t s) {
    SegPlan &pl = m->plan;
    if (pl.valid && pl.geo_uid == geo->uid && pl.tu == p.tu && pl.tv == p.tv &&
        pl.morton == p.morton && pl.channels == channels)
        return TETPROJ_OK;
    const int64_t budget = seg_chunk(channels);
    TP_CUDA(cudaStreamSynchronize(s));
    plan_free(pl);
    const int threads = p.tu * p.tv;
    const int64_t nblocks = (int64_t)p.g.na * p.tiles_u * p.tiles_v;
    pl.nrays = p.nrays;
    pl.nblocks = nblocks;
    cudaError_t e = dalloc(&pl.count, p.nrays, pl.bytes);
    if (e == cudaSuccess) e = dalloc(&pl.ray_off, p.nrays, pl.bytes);
    if (e == cudaSuccess) e = dalloc(&pl.block_cnt, nblocks, pl.bytes);
    if (e == cudaSuccess) e = dalloc(&pl.block_off, nblocks + 1, pl.bytes);
    if (e == cudaSuccess) e = dalloc(&pl.scan_tmp, scan_temp_elems(nblocks), pl.bytes);
    if (e == cudaSuccess) e = dalloc(&pl.counters, 1, pl.bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl.counters, 0, sizeof(DevCounters), s);
    if (e != cudaSuccess) { plan_free(pl); return cuda_status(e); }
    KParams pc = p;
    pc.m.counters = pl.counters;  // the user's statistics count only real calls
    pc.tr_tet = nullptr;
    pc.tr_len = nullptr;
    pc.tr_count = pl.count;
    pc.max_visits = 0;
    e = launch_walk(pc, TETPROJ_FILTERED, 1, MODE_TRACE, s);
    if (e == cudaSuccess) e = launch_block_offsets(pc, pl.count, pl.ray_off, pl.block_cnt, nblocks, s);
    if (e == cudaSuccess) e = launch_scan_i64(pl.block_cnt, pl.block_off, nblocks, pl.scan_tmp, s);
    std::vector<int64_t> off((size_t)nblocks + 1);
    DevCounters dc;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(off.data(), pl.block_off, sizeof(int64_t) * (nblocks + 1),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&dc, pl.counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { plan_free(pl); return cuda_status(e); }
    if (dc.error != 0) { int code = dc.error; plan_free(pl); return code; }
    // chunks: consecutive blocks, <= budget segments and <= q_cap rays
    const int64_t max_blocks = p.q_cap / threads;
    pl.chunk_b.push_back(0);
    pl.chunk_s.push_back(0);
    int64_t b0 = 0;
    while (b0 < nblocks) {
        int64_t b1 = b0 + 1;
        while (b1 < nblocks && b1 - b0 < max_blocks && off[b1 + 1] - off[b0] <= budget) ++b1;
        if (off[b1] - off[b0] > budget) { plan_free(pl); return TETPROJ_ERR_TOO_LARGE; }
        pl.chunk_b.push_back(b1);
        pl.chunk_s.push_back(off[b1]);
        if (off[b1] - off[b0] > pl.max_chunk) pl.max_chunk = off[b1] - off[b0];
        b0 = b1;
    }
    pl.geo_uid = geo->uid;
    pl.channels = channels;
    pl.tu = p.tu;
    pl.tv = p.tv;
    pl.morton = p.morton;
    pl.valid = true;
    return TETPROJ_OK;
}

// Sort buffers for nseg records: k[i] hold 8 bytes per record (C = 1 records,
// or C = 4 keys) and v[i] 16 bytes (C = 4 values); the buffer a sort does not
// end in is the run reduce's scratch.
static tetproj_status ensure_sort_ws(tetproj_mesh *m, int64_t nseg, int channels) {
    SortWs &w = m->sort;
    if (w.k[0] && w.cap >= nseg && w.cap_c >= channels) return TETPROJ_OK;
    cudaDeviceSynchronize();
    const int64_t cap = nseg > w.cap ? nseg : w.cap;
    const int cc = channels > w.cap_c ? channels : w.cap_c;
    sort_free(w);
    const int64_t hist = radix_hist_elems(cap);
    const int64_t tmp_h = scan_temp_elems(hist), tmp_r = scan_temp_elems(cap + 1);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = dalloc(&w.k[i], 2 * (cap + 1), w.bytes);
        if (e == cudaSuccess) e = dalloc(&w.v[i], cc == 4 ? 4 * (cap + 1) : 1, w.bytes);
    }
    if (e == cudaSuccess) e = dalloc(&w.hist, hist, w.bytes);
    if (e == cudaSuccess) e = dalloc(&w.tmp, tmp_h > tmp_r ? tmp_h : tmp_r, w.bytes);
    if (e != cudaSuccess) { sort_free(w); return cuda_status(e); }
    w.cap = cap;
    w.cap_c = cc;
    return TETPROJ_OK;
}

// mu_out = A^T y through the segment buffer: per chunk, the walk writes the
// chunk's segments, a stable radix sort groups them by tet, and one thread per
// tet sums its run in buffer order.  Deterministic.
static tetproj_status run_backward_sort(tetproj_mesh *m, const tetproj_geometry *geo, KParams &p,
                                        const tetproj_options &o, const void *y, void *mu_out,
                                        cudaStream_t s) {
    tetproj_status st = ensure_ws(m, o.precision, o.channels);
    if (st == TETPROJ_OK) st = attach_queue(m, p, o, s);
    if (st == TETPROJ_OK) st = ensure_plan(m, geo, p, o.channels, s);
    if (st == TETPROJ_OK) st = ensure_sort_ws(m, m->plan.max_chunk, o.channels);
    if (st != TETPROJ_OK) return st;
    const SegPlan &pl = m->plan;
    SortWs &w = m->sort;
    void *ws = m->ws[0][o.channels == 4];
    TP_CUDA(cudaMemsetAsync(ws, 0, (size_t)m->ws_bytes[0][o.channels == 4], s));
    int key_bits = 1;
    while ((int64_t(1) << key_bits) < m->nt) ++key_bits;
    p.in = y;
    p.out = ws;
    p.block_off = pl.block_off;
    p.ray_off = pl.ray_off;
    p.seg_key = w.k[0];
    p.seg_val = w.v[0];
    for (size_t c = 0; c + 1 < pl.chunk_b.size(); ++c) {
        const int64_t n = pl.chunk_s[c + 1] - pl.chunk_s[c];
        p.seg_base = pl.chunk_s[c];
        p.seg_cap = n;
        TP_CUDA(launch_walk_blocks(p, o.channels, MODE_SEG, pl.chunk_b[c], pl.chunk_b[c + 1], s));
        uint32_t *ko = nullptr;
        float *vo = nullptr;
        TP_CUDA(launch_radix_sort(w.k[0], w.v[0], w.k[1], w.v[1], n, o.channels, key_bits, w.hist,
                                  w.tmp, &ko, &vo, s));
        // scratch: the key buffer the sorted records are not in (2 (n + 1) words)
        uint32_t *scratch = ko == w.k[0] ? w.k[1] : w.k[0];
        TP_CUDA(launch_seg_reduce(ko, vo, n, o.channels, reinterpret_cast<float *>(ws), scratch,
                                  w.tmp, s));
    }
    TP_CUDA(launch_scatter_perm(m->perm, m->nt, o.channels, 0, ws, mu_out, s));
    return TETPROJ_OK;
}

tetproj_status tetproj_forward(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                               const void *mu, void *proj, const tetproj_options *opt,
                               void *stream) {
    if (!mesh || !geo || !mu || !proj) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    set_cone(p, geo);
    return run_forward(m, p, o, mu, proj, (cudaStream_t)stream, geo);
}

tetproj_status tetproj_backward(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                                const void *proj, void *mu_out, const tetproj_options *opt,
                                void *stream) {
    if (!mesh || !geo || !proj || !mu_out) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    set_cone(p, geo);
    if (o.scatter == TETPROJ_SCATTER_SORT) {
        if (o.precision != TETPROJ_FILTERED || rstar_unsupported(o) ||
            (o.flags & (TETPROJ_FLAG_ACC64 | TETPROJ_FLAG_ACC32)))
            return TETPROJ_ERR_ARG;
        return run_backward_sort(m, geo, p, o, proj, mu_out, (cudaStream_t)stream);
    }
    return run_backward(m, p, o, proj, mu_out, (cudaStream_t)stream, geo);
}

tetproj_status tetproj_forward_rays(const tetproj_mesh *mesh, const double *src,
                                    const double *dst, int64_t nrays, const void *mu, void *out,
                                    const tetproj_options *opt, void *stream) {
    if (!mesh || nrays < 0 || (nrays > 0 && (!src || !dst || !mu || !out))) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    if (nrays == 0) return TETPROJ_OK;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    p.src_kind = 1;
    p.rsrc = src;
    p.rdst = dst;
    p.nrays = nrays;
    return run_forward(m, p, o, mu, out, (cudaStream_t)stream);
}

tetproj_status tetproj_backward_rays(const tetproj_mesh *mesh, const double *src,
                                     const double *dst, int64_t nrays, const void *y,
                                     void *mu_out, const tetproj_options *opt, void *stream) {
    if (!mesh || nrays < 0 || !mu_out || (nrays > 0 && (!src || !dst || !y)))
        return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    if (o.scatter == TETPROJ_SCATTER_SORT) return TETPROJ_ERR_ARG;  // cone geometries only
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    p.src_kind = 1;
    p.rsrc = src;
    p.rdst = dst;
    p.nrays = nrays;
    if (nrays == 0) {
        TP_CUDA(cudaMemsetAsync(mu_out, 0,
                                (size_t)(m->nt * o.channels *
                                         (o.precision == TETPROJ_PLAIN_FP64 ? 8 : 4)),
                                (cudaStream_t)stream));
        return TETPROJ_OK;
    }
    return run_backward(m, p, o, y, mu_out, (cudaStream_t)stream);
}

tetproj_status tetproj_trace_rays(const tetproj_mesh *mesh, const double *src, const double *dst,
                                  int64_t nrays, int32_t max_visits, int32_t *out_tet,
                                  double *out_len, int32_t *out_count,
                                  const tetproj_options *opt, void *stream) {
    if (!mesh || nrays < 0 || max_visits < 0 ||
        (nrays > 0 && (!src || !dst || !out_count || (max_visits > 0 && (!out_tet || !out_len)))))
        return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    if (nrays == 0) return TETPROJ_OK;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    p.src_kind = 1;
    p.rsrc = src;
    p.rdst = dst;
    p.nrays = nrays;
    p.tr_tet = out_tet;
    p.tr_len = out_len;
    p.tr_count = out_count;
    p.max_visits = max_visits;
    if (rstar_unsupported(o)) return TETPROJ_ERR_ARG;
    st = attach_queue(m, p, o, (cudaStream_t)stream);
    if (st != TETPROJ_OK) return st;
    TP_CUDA(launch_walk(p, o.precision, 1, MODE_TRACE, (cudaStream_t)stream));
    return TETPROJ_OK;
}

tetproj_status tetproj_side_host(const double *S, const double *P, const double *p,
                                 const double *q, int64_t n, int8_t *sign, int8_t *stage) {
    if (n < 0 || (n > 0 && (!S || !P || !p || !q || !sign || !stage))) return TETPROJ_ERR_ARG;
    for (int64_t k = 0; k < n; ++k) {
        auto ld = [k](const double *a) { return mk(a[3 * k], a[3 * k + 1], a[3 * k + 2]); };
        int st = 0;
        int s = side_sign_cascade(ld(S), ld(P), ld(p), ld(q), &st);
        sign[k] = (int8_t)s;
        stage[k] = (int8_t)st;
    }
    return TETPROJ_OK;
}

tetproj_status tetproj_side_device(const double *S, const double *P, const double *p,
                                   const double *q, int64_t n, int8_t *sign, int8_t *stage,
                                   void *stream) {
    if (n < 0 || (n > 0 && (!S || !P || !p || !q || !sign || !stage))) return TETPROJ_ERR_ARG;
    TP_CUDA(launch_side_device(S, P, p, q, n, sign, stage, (cudaStream_t)stream));
    return TETPROJ_OK;
}

}  // extern "C"

// ------------------------------------------------ allocation-free backprojection
//
// tetproj_backward_noalloc computes what tetproj_backward computes, with the
// same accumulator (FP64 at C = 1 on the filtered path, two-level FP32 -> FP64
// for dense problems, FP32 otherwise, FP64 on the plain path), for callers
// that cannot call cudaMalloc at that point -- for instance code whose device
// memory is entirely owned by another allocator (a framework's caching pool
// that has already reserved the device), or a latency-critical loop that must
// not pay cudaMalloc's implicit device synchronisation.  tetproj_backward
// allocates the mesh's workspace on its first call; this variant instead uses
// the file-scope device array below, so it never allocates or frees anything.
//
// Its scratch is the tet-ordered accumulator (up to kNoAllocAccBytes; the
// two-level case holds the FP32 and the FP64 accumulator side by side) and
// the deferral queue of the filtered walk with its crossing fixes
// (kNoAllocQueue entries; launches are chunked to fit it).  The array is part
// of the library image, so every GPU that loads libtetproj.so holds it (52 MB)
// until the process exits.
// Every call shares it and it keeps the previous call's contents: the
// accumulators are cleared at the start of each call, and calls that overlap
// on the GPU (different streams, no ordering) race on it.
static const int64_t kNoAllocAccBytes = TETPROJ_NOALLOC_ACC_BYTES;
static_assert(kNoAllocAccBytes % 256 == 0, "accumulator region keeps the queue 256-byte aligned");
static const int64_t kNoAllocQueue = int64_t(1) << 18;
static const int64_t kNoAllocQueueBytes = ((int64_t)kNoAllocQueue * (int64_t)sizeof(QEntry) +
                                           ((int64_t)kNoAllocQueue / 2) * (int64_t)sizeof(XFix));
static const int64_t kNoAllocBytes = kNoAllocAccBytes + kNoAllocQueueBytes + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
struct NoAllocAddr {
    void *addr;
    unsigned long long ctx;  // cuCtxGetId of the context the address belongs to; 0 unknown
};
static NoAllocAddr g_noalloc_addr[128] = {};

// Unique id of the calling thread's current CUDA context (0 when there is none
// or the driver does not export the query).  Resolved through the runtime's
// driver entry points, so the library does not link libcuda itself.
static unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached together with the id of the
// context it belongs to.  A new context on the device (after cudaDeviceReset,
// or a primary context released and created again) reloads the module, so the
// address is looked up again when the id changes; when the id cannot be read
// it is looked up on every call.
static tetproj_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return TETPROJ_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocAddr &slot = g_noalloc_addr[dev];
    const unsigned long long ctx = current_context_id();
    if (!slot.addr || ctx == 0 || ctx != slot.ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        slot.addr = p;
        slot.ctx = current_context_id();  // the lookup makes the primary context current
    }
    *out = static_cast<unsigned char *>(slot.addr);
    return TETPROJ_OK;
}

static int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

extern "C" tetproj_status tetproj_backward_noalloc(const tetproj_mesh *mesh,
                                                   const tetproj_geometry *geo, const void *proj,
                                                   void *mu_out, const tetproj_options *opt,
                                                   void *stream) {
    if (!mesh || !geo || !proj || !mu_out) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    // the sort-and-reduce scatter needs buffers sized by the segment count
    if (o.scatter == TETPROJ_SCATTER_SORT || rstar_unsupported(o)) return TETPROJ_ERR_ARG;
    if ((o.flags & TETPROJ_FLAG_ACC64) && o.precision == TETPROJ_FILTERED &&
        o.scatter == TETPROJ_SCATTER_SORT)
        return TETPROJ_ERR_ARG;  // FP64 accumulation is an atomic-scatter variant
    const int f64 = o.precision == TETPROJ_PLAIN_FP64;
    KParams p = base_params(mesh, o);
    set_cone(p, geo);
    // the accumulator tetproj_backward would use
    const int64_t n = mesh->nt * o.channels;
    const bool acc64 = use_acc64(o);
    const bool two_level = !f64 && !acc64 && !(o.flags & TETPROJ_FLAG_ACC32) &&
                           dense_acc(mesh->nt, o.channels, p.nrays);
    const int64_t off64 = two_level ? align256(4 * n) : 0;
    const int64_t need = (f64 || acc64) ? 8 * n : (two_level ? off64 + 8 * n : 4 * n);
    if (need > kNoAllocAccBytes) return TETPROJ_ERR_TOO_LARGE;
    unsigned char *base = nullptr;
    st = noalloc_scratch(&base);
    if (st != TETPROJ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!f64) {
        p.q = reinterpret_cast<QEntry *>(base + kNoAllocAccBytes);
        p.q_count = reinterpret_cast<unsigned long long *>(
            base + kNoAllocAccBytes + kNoAllocQueueBytes);
        p.q_cap = kNoAllocQueue;
    }
    p.in = proj;
    p.out = base;
    TP_CUDA(cudaMemsetAsync(base, 0, (size_t)need, s));
    if (f64) {
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD, s));
        TP_CUDA(launch_scatter_perm(mesh->perm, mesh->nt, o.channels, 1, base, mu_out, s));
    } else if (acc64) {
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD64, s));
        TP_CUDA(launch_scatter_perm_d2f(mesh->perm, mesh->nt, o.channels,
                                        reinterpret_cast<const double *>(base),
                                        reinterpret_cast<float *>(mu_out), s));
    } else if (two_level) {
        AccMerge mg{reinterpret_cast<float *>(base), reinterpret_cast<double *>(base + off64), n,
                    dense_chunk_rays(mesh->nt)};
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD, s, nullptr, &mg));
        TP_CUDA(launch_scatter_perm_d2f(mesh->perm, mesh->nt, o.channels,
                                        reinterpret_cast<const double *>(base + off64),
                                        reinterpret_cast<float *>(mu_out), s));
    } else {
        TP_CUDA(launch_walk(p, o.precision, o.channels, MODE_BWD, s));
        TP_CUDA(launch_scatter_perm(mesh->perm, mesh->nt, o.channels, 0, base, mu_out, s));
    }
    return TETPROJ_OK;
}

// ------------------------------------------------------------ batched calls
//
// A batch holds many (mesh, geometry) problems of uneven size and runs their
// forward or backward projections in one persistent work-queue launch per
// round (kernels.cu: k_batch32 / k_batch_resume32).  Operand buffers are bound
// once (tetproj_batch_bind) so that forward/backward take only a stream and
// can be captured in a CUDA graph and replayed.

// BVH nodes each warp of the batched kernel stages in shared memory
static const int kBatchWarpNodes = 0;

struct tetproj_batch {
    int n = 0, channels = 1;
    std::vector<KParams> base;        // per-problem parameters (no operands)
    std::vector<const tetproj_mesh *> meshes;
    std::vector<void *> ws_in, ws_acc;
    std::vector<int64_t> ws_bytes;
    std::vector<int64_t> item_begin;  // host copy, n + 1 entries
    std::vector<const void *> mu, y;
    std::vector<void *> proj, mu_out;
    BatchProblem *d_fwd = nullptr, *d_bwd = nullptr;
    int64_t *d_item_begin = nullptr;
    QEntry *q = nullptr;
    unsigned long long *q_count = nullptr;
    unsigned *item_counter = nullptr;
    int64_t q_cap = 0;
    int smem_nodes = 64;
    unsigned grid_fwd = 0, grid_bwd = 0, rgrid = 0;
    bool acc64 = false;  // C = 1: FP64 accumulators (atomic or warp-aggregated per problem)
    bool bound = false;
    ResumeOverlap ov{};  // second queue + auxiliary stream when there are several rounds
    bool ov_ready = false;
    // dense problems at C = 4: FP32 scratch the walk reduces into, merged into
    // the FP64 accumulator (ws_acc) after every round
    std::vector<float *> acc32;   // per problem, null unless dense
    std::vector<AccMerge> merges; // the dense problems' merges
    std::vector<int64_t> cuts;    // backprojection rounds (item boundaries; empty: uniform)
    BatchWait wait{kBatchWaitPolls, 0};  // bounded waits of the persistent kernel
    // entry maps per round (forward: uniform rounds, backward: `cuts` or uniform)
    int32_t *emap = nullptr;
    EmapView *d_views[2] = {nullptr, nullptr};
    std::vector<BatchEmapRound> em_rounds[2];
    std::vector<BatchEmapJob> em_jobs[2];
    BatchEmap em[2] = {};
    bool em_ready = false;
};

static void batch_free(tetproj_batch *b) {
    if (!b) return;
    for (void *p : b->ws_in) cudaFree(p);
    for (void *p : b->ws_acc) cudaFree(p);
    for (float *p : b->acc32) cudaFree(p);
    cudaFree(b->d_fwd);
    cudaFree(b->d_bwd);
    cudaFree(b->d_item_begin);
    cudaFree(b->q);
    cudaFree(b->q_count);
    cudaFree(b->item_counter);
    if (b->ov_ready) overlap_release(b->ov);
    cudaFree(b->emap);
    cudaFree(b->d_views[0]);
    cudaFree(b->d_views[1]);
    delete b;
}

// Entry maps of the batched launch (the single-problem walk's, per round):
// for every round, the angles of each problem with items in it are drawn
// into one buffer before the round's walk.  Problems whose source circle is
// not outside their mesh's bounding sphere get no map.  Rounds are the
// launch's: uniform for the forward, `cuts` (when set) for the backward.
static cudaError_t batch_entry_maps(tetproj_batch *b, const tetproj_geometry *const *geos) {
    const int n = b->n;
    const int64_t total = b->item_begin.back();
    const int64_t ri = batch_round_items(b->q_cap);
    if (ri < 1) return cudaSuccess;
    std::vector<int64_t> uni;
    for (int64_t r = 0; r < total; r += ri) uni.push_back(r);
    uni.push_back(total);
    const std::vector<int64_t> *bounds[2] = {&uni, b->cuts.empty() ? &uni : &b->cuts};
    std::vector<char> ok(n);
    for (int k = 0; k < n; ++k)
        ok[k] = b->base[k].entry == ENTRY_BVH && geos[k]->dso > 1.75 * (double)b->meshes[k]->radius;
    int64_t maxlen = 0;
    std::vector<std::vector<EmapView>> views(2);
    for (int d = 0; d < 2; ++d) {
        const std::vector<int64_t> &B = *bounds[d];
        const int64_t nr = (int64_t)B.size() - 1;
        views[d].assign((size_t)(nr * n), EmapView{nullptr, 0, 0});
        for (int64_t i = 0; i < nr; ++i) {
            BatchEmapRound R{(int32_t)b->em_jobs[d].size(), 0, 0};
            for (int k = 0; k < n; ++k) {
                const int64_t i0 = b->item_begin[k], i1 = b->item_begin[k + 1];
                if (!ok[k] || i1 <= B[i] || i0 >= B[i + 1]) continue;
                const KParams &P = b->base[k];
                const int wpt_log = P.log_tu + P.log_tv - 5;
                const int64_t per = (int64_t)P.tiles_u * P.tiles_v, nblk = (int64_t)P.g.na * per;
                const int64_t lo = (B[i] > i0 ? B[i] : i0) - i0, hi = (B[i + 1] < i1 ? B[i + 1] : i1) - i0 - 1;
                const int64_t b_lo = lo >> wpt_log;
                int64_t b_hi = hi >> wpt_log;
                if (b_lo >= nblk) continue;  // only the padding of the problem's last chunk
                if (b_hi >= nblk) b_hi = nblk - 1;
                const int64_t a_lo = b_lo / per, na = b_hi / per - a_lo + 1;
                if (na > 65535) continue;
                const int64_t pix = (int64_t)P.g.nu * P.g.nv;
                b->em_jobs[d].push_back(BatchEmapJob{k, (int32_t)a_lo, (int32_t)na, R.len});
                // the view's pointer is the offset for now
                views[d][(size_t)(i * n + k)] = EmapView{reinterpret_cast<const int32_t *>(R.len),
                                                         a_lo * pix, na * pix};
                R.len += na * pix;
                ++R.count;
            }
            b->em_rounds[d].push_back(R);
            if (R.len > maxlen) maxlen = R.len;
        }
    }
    if (maxlen == 0 || maxlen > (int64_t(1) << 27)) return cudaSuccess;  // no map (or > 512 MB)
    cudaError_t e = cudaMalloc((void **)&b->emap, (size_t)maxlen * sizeof(int32_t));
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        for (EmapView &v : views[d])
            if (v.len > 0) v.emap = b->emap + reinterpret_cast<intptr_t>(v.emap);
        e = cudaMalloc((void **)&b->d_views[d], sizeof(EmapView) * views[d].size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_views[d], views[d].data(), sizeof(EmapView) * views[d].size(),
                           cudaMemcpyHostToDevice);
        b->em[d] = BatchEmap{b->emap, b->d_views[d], b->em_rounds[d].data(), b->em_jobs[d].data(),
                             b->base.data(), n};
    }
    if (e != cudaSuccess) return e;
    b->em_ready = true;
    return cudaSuccess;
}

extern "C" tetproj_status tetproj_batch_create(const tetproj_mesh *const *meshes,
                                               const tetproj_geometry *const *geos,
                                               const int32_t *tiles, int32_t n,
                                               int32_t channels, tetproj_batch **out) {
    if (!out) return TETPROJ_ERR_ARG;
    *out = nullptr;
    if (!meshes || !geos || n < 1 || n >= (1 << 20) || (channels != 1 && channels != 4))
        return TETPROJ_ERR_ARG;
    tetproj_batch *b = new (std::nothrow) tetproj_batch();
    if (!b) return TETPROJ_ERR_OOM;
    b->n = n;
    b->channels = channels;
    b->acc64 = channels == 1;
    b->item_begin.assign(1, 0);
    int64_t total_rays = 0;
    for (int k = 0; k < n; ++k) {
        if (!meshes[k] || !geos[k]) { batch_free(b); return TETPROJ_ERR_ARG; }
        tetproj_options o;
        tetproj_default_options(&o);
        o.channels = channels;
        if (tiles) {
            o.tile_u = tiles[4 * k];
            o.tile_v = tiles[4 * k + 1];
            o.order = tiles[4 * k + 2];
            o.scatter = tiles[4 * k + 3];
        }
        tetproj_options oo;
        tetproj_status st = check_opts(&o, oo);
        if (st == TETPROJ_OK && (oo.scatter == TETPROJ_SCATTER_SORT || rstar_unsupported(oo)))
            st = TETPROJ_ERR_ARG;
        if (st != TETPROJ_OK) { batch_free(b); return st; }
        KParams p = base_params(meshes[k], oo);
        set_cone(p, geos[k]);
        b->base.push_back(p);
        b->meshes.push_back(meshes[k]);
        // warp items: 32 in-tile threads of one tile (tiles hold 32..256 threads),
        // padded to whole chunks so that every problem starts a chunk
        int64_t items = (int64_t)p.g.na * p.tiles_u * p.tiles_v * ((oo.tile_u * oo.tile_v) / 32);
        items = (items + kBatchChunk - 1) / kBatchChunk * kBatchChunk;
        if (items >= (int64_t(1) << 31)) { batch_free(b); return TETPROJ_ERR_TOO_LARGE; }
        b->item_begin.push_back(b->item_begin.back() + items);
        total_rays += items * 32;
        int64_t bytes = meshes[k]->nt * channels * 4;
        void *a = nullptr, *c = nullptr;
        cudaError_t e = cudaMalloc(&a, (size_t)bytes);
        // accumulator: sized for FP64 (the FP32 case uses the first half)
        if (e == cudaSuccess) e = cudaMalloc(&c, (size_t)(2 * bytes));
        b->ws_in.push_back(a);
        b->ws_acc.push_back(c);
        b->ws_bytes.push_back(bytes);
        float *s32 = nullptr;
        const int64_t prays = (int64_t)p.g.na * p.g.nu * p.g.nv;
        if (e == cudaSuccess && channels == 4 && dense_acc(meshes[k]->nt, channels, prays))
            e = cudaMalloc((void **)&s32, (size_t)bytes);
        b->acc32.push_back(s32);
        if (e != cudaSuccess) { batch_free(b); return cuda_status(e); }
    }
    if (b->item_begin.back() >= (int64_t(1) << 40)) { batch_free(b); return TETPROJ_ERR_TOO_LARGE; }
    int64_t need = total_rays < kBatchQueueMax ? total_rays : kBatchQueueMax;
    need = ((need + 4095) / 4096) * 4096;
    cudaError_t e = cudaMalloc((void **)&b->q, (size_t)queue_bytes(need));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->q_count, kQueueCountBytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->item_counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_fwd, sizeof(BatchProblem) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_bwd, sizeof(BatchProblem) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_item_begin, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_item_begin, b->item_begin.data(), sizeof(int64_t) * (n + 1),
                       cudaMemcpyHostToDevice);
    // several rounds: round r's resume overlaps round r + 1's walk
    if (e == cudaSuccess && total_rays > kBatchQueueMax) {
        e = overlap_create(b->ov, need);
        b->ov_ready = e == cudaSuccess;
    }
    if (e != cudaSuccess) { batch_free(b); return cuda_status(e); }
    b->q_cap = need;
    // Backprojection rounds: uniform rounds at the queue capacity, cut further
    // inside dense problems only, so that each merge interval holds at most
    // dense_chunk_rays of a dense problem (uniformly shorter rounds would add
    // a persistent launch tail to every round of every problem: measured
    // +40% on the backprojection of 24 problems).
    for (int k = 0; k < n; ++k)
        if (b->acc32[k])
            b->merges.push_back(AccMerge{b->acc32[k], reinterpret_cast<double *>(b->ws_acc[k]),
                                         meshes[k]->nt * channels, 0});
    if (!b->merges.empty()) {
        // greedy: each round ends at the queue capacity or where a dense
        // problem would exceed its merge interval inside the round
        const int64_t total = b->item_begin.back();
        const int64_t round_items = (need / (32 * kBatchChunk)) * kBatchChunk;
        std::vector<int64_t> step(n, 0);
        for (int k = 0; k < n; ++k)
            if (b->acc32[k]) {
                step[k] = dense_chunk_rays(meshes[k]->nt) / (32 * kBatchChunk) * kBatchChunk;
                if (step[k] < kBatchChunk) step[k] = kBatchChunk;
            }
        for (int64_t r = 0; r < total;) {
            int64_t e = total - r < round_items ? total : r + round_items;
            for (int k = 0; k < n; ++k) {
                const int64_t b0 = b->item_begin[k], b1 = b->item_begin[k + 1];
                if (!step[k] || b1 <= r || b0 >= e) continue;
                const int64_t lim = (b0 > r ? b0 : r) + step[k];
                if (lim < e && lim < b1) e = lim;
            }
            b->cuts.push_back(r);
            r = e;
        }
        b->cuts.push_back(total);
    }
    // launch shapes are fixed here so that forward/backward issue stream work only
    int snodes = 0;
    for (auto &p : b->base) snodes = p.smem_nodes > snodes ? p.smem_nodes : snodes;
    b->smem_nodes = snodes < kBatchWarpNodes ? snodes : kBatchWarpNodes;
    e = batch_grid(channels, MODE_FWD, b->smem_nodes, b->grid_fwd);
    if (e == cudaSuccess)
        e = batch_grid(channels, b->acc64 ? MODE_BWD64 : MODE_BWD, b->smem_nodes, b->grid_bwd);
    if (e != cudaSuccess) { batch_free(b); return cuda_status(e); }
    b->rgrid = (unsigned)(4 * device_sm_count());
    for (auto &p : b->base) {
        p.q = b->q;
        p.q_count = b->q_count;
        p.q_cap = b->q_cap;
    }
    b->mu.assign(n, nullptr);
    b->y.assign(n, nullptr);
    b->proj.assign(n, nullptr);
    b->mu_out.assign(n, nullptr);
    e = batch_entry_maps(b, geos);
    if (e != cudaSuccess) { batch_free(b); return cuda_status(e); }
    *out = b;
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_batch_bind(tetproj_batch *b, const void *const *mu,
                                             void *const *proj, const void *const *y,
                                             void *const *mu_out) {
    if (!b) return TETPROJ_ERR_ARG;
    std::vector<BatchProblem> f(b->n), g(b->n);
    for (int k = 0; k < b->n; ++k) {
        b->mu[k] = mu ? mu[k] : nullptr;
        b->proj[k] = proj ? proj[k] : nullptr;
        b->y[k] = y ? y[k] : nullptr;
        b->mu_out[k] = mu_out ? mu_out[k] : nullptr;
        std::memset(&f[k], 0, sizeof(BatchProblem));
        std::memset(&g[k], 0, sizeof(BatchProblem));
        f[k].p = b->base[k];
        f[k].p.in = b->ws_in[k];
        f[k].p.out = b->proj[k];
        f[k].p.qtag = (int64_t)k << 40;
        g[k].p = b->base[k];
        g[k].p.in = b->y[k];
        g[k].p.out = b->acc32[k] ? (void *)b->acc32[k] : b->ws_acc[k];
        g[k].p.qtag = (int64_t)k << 40;
    }
    TP_CUDA(cudaMemcpy(b->d_fwd, f.data(), sizeof(BatchProblem) * b->n, cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(b->d_bwd, g.data(), sizeof(BatchProblem) * b->n, cudaMemcpyHostToDevice));
    b->bound = true;
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_batch_forward(tetproj_batch *b, void *stream) {
    if (!b || !b->bound) return TETPROJ_ERR_ARG;
    for (int k = 0; k < b->n; ++k)
        if (!b->mu[k] || !b->proj[k]) return TETPROJ_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < b->n; ++k)
        TP_CUDA(launch_gather_perm(b->meshes[k]->perm, b->meshes[k]->nt, b->channels, 0, b->mu[k],
                                   b->ws_in[k], s));
    TP_CUDA(launch_batch(b->d_fwd, b->d_item_begin, b->n, b->item_begin.back(),
                         b->channels, MODE_FWD, b->grid_fwd, b->rgrid, b->q, b->q_count, b->q_cap, b->item_counter,
                         b->smem_nodes, s, b->ov_ready ? &b->ov : nullptr, nullptr, 0, nullptr, 0,
                         b->wait, b->em_ready ? &b->em[0] : nullptr));
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_batch_backward(tetproj_batch *b, void *stream) {
    if (!b || !b->bound) return TETPROJ_ERR_ARG;
    for (int k = 0; k < b->n; ++k)
        if (!b->y[k] || !b->mu_out[k]) return TETPROJ_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < b->n; ++k) {
        const bool wide = b->acc64 || b->acc32[k];
        TP_CUDA(cudaMemsetAsync(b->ws_acc[k], 0, (size_t)(wide ? 2 : 1) * b->ws_bytes[k], s));
        if (b->acc32[k]) TP_CUDA(cudaMemsetAsync(b->acc32[k], 0, (size_t)b->ws_bytes[k], s));
    }
    TP_CUDA(launch_batch(b->d_bwd, b->d_item_begin, b->n, b->item_begin.back(),
                         b->channels, b->acc64 ? MODE_BWD64 : MODE_BWD, b->grid_bwd, b->rgrid, b->q, b->q_count, b->q_cap, b->item_counter,
                         b->smem_nodes, s, b->ov_ready ? &b->ov : nullptr,
                         b->cuts.empty() ? nullptr : b->cuts.data(), (int)b->cuts.size(),
                         b->merges.empty() ? nullptr : b->merges.data(), (int)b->merges.size(),
                         b->wait, b->em_ready ? &b->em[1] : nullptr));
    for (int k = 0; k < b->n; ++k) {
        if (b->acc64 || b->acc32[k])
            TP_CUDA(launch_scatter_perm_d2f(b->meshes[k]->perm, b->meshes[k]->nt, b->channels,
                                            reinterpret_cast<const double *>(b->ws_acc[k]),
                                            reinterpret_cast<float *>(b->mu_out[k]), s));
        else
            TP_CUDA(launch_scatter_perm(b->meshes[k]->perm, b->meshes[k]->nt, b->channels, 0,
                                        b->ws_acc[k], b->mu_out[k], s));
    }
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_batch_set_wait(tetproj_batch *b, int32_t max_polls,
                                                 int32_t never_satisfied) {
    if (!b || max_polls < 0) return TETPROJ_ERR_ARG;
    b->wait.limit = max_polls == 0 ? kBatchWaitPolls : max_polls;
    b->wait.offset = never_satisfied ? (1 << 30) : 0;
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_batch_destroy(tetproj_batch *b) {
    if (!b) return TETPROJ_ERR_ARG;
    cudaDeviceSynchronize();
    batch_free(b);
    return TETPROJ_OK;
}

// ------------------------------------------------- the paper's walk (Alg. 1-2)

static tetproj_status run_forward_mt(tetproj_mesh *m, KParams &p, const tetproj_options &o,
                                     const void *mu, void *out, int8_t *status, cudaStream_t s) {
    if (o.channels != 1 || rstar_unsupported(o)) return TETPROJ_ERR_ARG;
    if (p.src_kind == 0 && o.tile_u * o.tile_v > 128) return TETPROJ_ERR_ARG;
    tetproj_status st = ensure_ws(m, o.precision, 1);
    if (st != TETPROJ_OK) return st;
    const int f64 = o.precision == TETPROJ_PLAIN_FP64;
    void *ws = m->ws[f64][0];
    TP_CUDA(launch_gather_perm(m->perm, m->nt, 1, f64, mu, ws, s));
    p.in = ws;
    p.out = out;
    TP_CUDA(launch_walk_mt(p, f64, status, s));
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_forward_mt(const tetproj_mesh *mesh,
                                             const tetproj_geometry *geo, const void *mu,
                                             void *proj, int8_t *status,
                                             const tetproj_options *opt, void *stream) {
    if (!mesh || !geo || !mu || !proj) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    set_cone(p, geo);
    return run_forward_mt(m, p, o, mu, proj, status, (cudaStream_t)stream);
}

extern "C" tetproj_status tetproj_forward_rays_mt(const tetproj_mesh *mesh, const double *src,
                                                  const double *dst, int64_t nrays,
                                                  const void *mu, void *out, int8_t *status,
                                                  const tetproj_options *opt, void *stream) {
    if (!mesh || nrays < 0 || (nrays > 0 && (!src || !dst || !mu || !out))) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    if (nrays == 0) return TETPROJ_OK;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    p.src_kind = 1;
    p.rsrc = src;
    p.rdst = dst;
    p.nrays = nrays;
    return run_forward_mt(m, p, o, mu, out, status, (cudaStream_t)stream);
}

// ------------------------------------------------------------ entry search

extern "C" tetproj_status tetproj_entry(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                                        int32_t *entry_tet, const tetproj_options *opt,
                                        void *stream) {
    if (!mesh || !geo || !entry_tet) return TETPROJ_ERR_ARG;
    tetproj_options o;
    tetproj_status st = check_opts(opt, o);
    if (st != TETPROJ_OK) return st;
    if (o.precision != TETPROJ_FILTERED) return TETPROJ_ERR_ARG;
    o.channels = 1;
    tetproj_mesh *m = const_cast<tetproj_mesh *>(mesh);
    KParams p = base_params(m, o);
    set_cone(p, geo);
    if (p.entry == ENTRY_RSTAR) st = ensure_rstar(m, p);
    if (st == TETPROJ_OK) st = attach_queue(m, p, o, (cudaStream_t)stream);
    if (st != TETPROJ_OK) return st;
    p.tr_count = entry_tet;
    TP_CUDA(launch_walk(p, TETPROJ_FILTERED, 1, MODE_ENTRY, (cudaStream_t)stream));
    return TETPROJ_OK;
}

extern "C" tetproj_status tetproj_rstar_build_host(const double *vertices, int64_t nv,
                                                   const int32_t *tets, int64_t nt,
                                                   tetproj_rstar_info *out) {
    if (!out) return TETPROJ_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    HostMesh H;
    tetproj_status st = build_host_mesh(vertices, nv, tets, nt, H);
    if (st != TETPROJ_OK) return st;
    std::vector<RStarNode> nodes;
    rstar_build(H.bfaces, nodes);
    RStarStats rs = rstar_check(H.bfaces, nodes);
    out->nodes = rs.nodes;
    out->leaves = rs.leaves;
    out->entries = rs.entries;
    out->depth = rs.depth;
    out->min_fill = rs.min_fill;
    out->max_fill = rs.max_fill;
    out->ok = rs.ok;
    return TETPROJ_OK;
}
