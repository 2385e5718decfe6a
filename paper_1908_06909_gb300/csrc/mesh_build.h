// mesh_build.h -- host-side mesh preprocessing (see mesh_build.cpp).
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/tetproj.h"
#include "tetproj_internal.h"

namespace tp {

struct HostMesh {
    std::vector<TetRec32> rec32;
    std::vector<TetRec64> rec64;
    std::vector<BvhNode> bvh;
    std::vector<BFace32> bfaces;
    std::vector<int32_t> perm;  // h -> user tet id
    std::vector<int4> vid;      // h -> user vertex ids in local (oriented) order
    int32_t root = 0;
    float radius = 0.f;
    double bbox[6] = {0, 0, 0, 0, 0, 0};
    int64_t nt = 0, nv = 0, nb = 0, nflipped = 0;
};

tetproj_status build_host_mesh(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                               HostMesh &M);
tetproj_status topology_host(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                             int32_t *adj_out, int64_t *nboundary, int64_t *nflipped);

}  // namespace tp
