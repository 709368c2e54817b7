// blockindex.h -- 2D voxel blocks of the map and a KD-tree over their centres
// (Sec. III-B.2 of 3DGS-ReLoc: the map is divided into a 2D voxel grid, each
// voxel has a unique hash ID, and a KD-tree built from the voxel centres
// answers "which voxels lie within range of this camera").
#pragma once
#include <cstdint>
#include <vector>

namespace reloc {

struct BlockIndex {
    double B = 20.0;                       // block edge, metres
    std::vector<int64_t> bx, by;           // block coordinates, ascending (bx, by)
    std::vector<int64_t> begin, end;       // [begin, end) in the block-ordered map
    std::vector<double> cx, cy;            // block centres
    std::vector<int> kd;                   // implicit KD-tree: node -> block id

    // Partition n means (xyz float triples) into blocks of edge B.  order
    // receives the block order: order[p] = original index of the Gaussian at
    // block-ordered position p (stable: index order inside a block).
    void build(const float *means, int64_t n, double B, std::vector<int64_t> &order);

    // Ids of every block whose centre is within r of (x, y), ascending.
    void range(double x, double y, double r, std::vector<int> &out) const;

    size_t size() const { return bx.size(); }
};

}  // namespace reloc
