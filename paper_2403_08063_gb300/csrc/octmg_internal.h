// Internal declarations shared by the host forest builder and the CUDA solver.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "octmg.h"

namespace octmg {

// One ghost face of a block that is filled from a single source block (Sec. 3.1): the domain boundary,
// a same-level neighbour, or (C2F, Sec. 3.3.2) the coarser neighbour whose face segment (seg1, seg2) it touches.
enum FaceKind : int8_t { FK_BND = 0, FK_SAME = 1, FK_C2F = 2 };

struct FaceItem {
    int32_t blk;   // block whose ghost face is written
    int32_t nbr;   // source block (same level or coarser); -1 for the boundary
    int8_t axis;   // 0 = x, 1 = y, 2 = z
    int8_t side;   // 0 = minus face, 1 = plus face
    int8_t kind;   // FaceKind
    int8_t seg1;   // C2F: which half of the coarse face along the first tangential axis
    int8_t seg2;   // C2F: same along the second tangential axis
    int8_t pad[3];
};
static_assert(sizeof(FaceItem) == 16, "FaceItem layout");

// One quarter of a coarse block's face whose four finer neighbours each fill a segment of its ghosts (F2C,
// Sec. 3.3.1; N_neigh = r^(D-1) = 4 segments, Sec. 3.1).
struct SegItem {
    int32_t coarse;  // coarse block whose ghost segment is written (its face (axis, side))
    int32_t fine;    // the finer neighbour covering segment (s1, s2)
    int8_t axis, side, s1, s2;
};
static_assert(sizeof(SegItem) == 12, "SegItem layout");

// How the blocks of level l+1 come from level l: halving a block (same key, n/2), merging a complete octet of
// 4^3 siblings into their parent, or carrying a block over unchanged.
enum XferKind : int32_t { XF_HALVE = 0, XF_MERGE = 1, XF_COPY = 2 };
struct XferItem {
    int32_t kind;
    int32_t src[8];  // level-l blocks: HALVE/COPY use src[0]; MERGE: child of octant (a + 2b + 4c)
};

// A block of problem p: (level, i, j, k) covers [i, i+1] x [j, j+1] x [k, k+1] / (R 2^level) of that problem's
// unit cube.  Problems are independent forests solved together.
struct Key {
    int32_t p, lev, i, j, k;
    bool operator==(const Key &o) const { return p == o.p && lev == o.lev && i == o.i && j == o.j && k == o.k; }
};

// One edge (12 per block) or corner (8 per block) of a block's ghost layer, for the edge and corner ghosts the
// trilinear prolongation reads.  Edges: code = 4 q + bits, q = 0 for the (x, y) edge, 1 for (x, z), 2 for (y, z),
// bit 0 set for the plus side of the first axis, bit 1 for the second.  Corners: code = bits, bit a set for the plus
// side of axis a.  nbr: the same-level block across the edge or corner (the same problem), -1 if there is none (the
// ghosts are then extrapolated from the block's own face or edge ghosts).
struct DiagItem {
    int32_t blk, nbr, code, pad;
};
static_assert(sizeof(DiagItem) == 16, "DiagItem layout");

struct HostLevel {
    int32_t n = 0;
    std::vector<Key> keys;
    std::vector<double> h;          // cell width per block
    std::vector<FaceItem> faces;    // every block face that is not a coarse side of a refinement interface
    std::vector<SegItem> segs;      // coarse sides of refinement interfaces, 4 segments each
    std::vector<XferItem> to_next;  // per block of level l+1 (empty on the coarsest level)
    std::vector<DiagItem> edges, corners;  // filled by build_diagonal (trilinear prolongation only)
};

struct HostHierarchy {
    int32_t R = 0;
    std::vector<HostLevel> levels;
};

// Builds the hierarchy of n_problems independent forests sharing R and n; returns MG_OK or an error with a message.
// Below 4^3, problems whose level still has more than max_coarse unknowns merge their deepest complete octets;
// the others carry their blocks over unchanged.
mg_status build_hierarchy(int32_t R, int32_t n, int32_t n_problems, const std::vector<Key> &leaves,
                          int32_t max_coarse, HostHierarchy &out, std::string &err);

// Edge and corner items of every block of a level (see DiagItem).
void build_diagonal(int32_t R, HostLevel &L);

void set_error(const std::string &msg);

}  // namespace octmg
