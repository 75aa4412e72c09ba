// Host side of the forest: leaf validation, neighbour / segment tables (Sec. 3.1), and the multigrid hierarchy
// (block-local halving down to 4^3 cells per block, Sec. 5, then merging of complete sibling octets).
#include <algorithm>
#include <cmath>
#include <unordered_map>

#include "octmg_internal.h"

namespace octmg {
namespace {

struct KeyHash {
    size_t operator()(const Key &k) const {
        uint64_t h = static_cast<uint64_t>(k.p) * 0x100000001B3ull + static_cast<uint64_t>(k.lev + 64);
        h = h * 0x9E3779B97F4A7C15ull ^ static_cast<uint32_t>(k.i);
        h = h * 0x9E3779B97F4A7C15ull ^ static_cast<uint32_t>(k.j);
        h = h * 0x9E3779B97F4A7C15ull ^ static_cast<uint32_t>(k.k);
        return static_cast<size_t>(h ^ (h >> 29));
    }
};
using KeyMap = std::unordered_map<Key, int32_t, KeyHash>;

// Blocks per axis at a level: R * 2^lev (negative levels group roots 2x2x2); false if not a whole number >= 1.
bool blocks_per_axis(int32_t R, int32_t lev, int64_t &m) {
    if (lev >= 0) {
        if (lev > 40) return false;
        m = static_cast<int64_t>(R) << lev;
        return true;
    }
    int32_t d = -lev;
    if (d > 30 || (R % (1 << d)) != 0) return false;
    m = R >> d;
    return m >= 1;
}

int coord(const Key &k, int axis) { return axis == 0 ? k.i : (axis == 1 ? k.j : k.k); }
void set_coord(Key &k, int axis, int v) {
    if (axis == 0) k.i = v; else if (axis == 1) k.j = v; else k.k = v;
}
void tangential(int axis, int &t1, int &t2) {
    t1 = axis == 0 ? 1 : 0;
    t2 = axis == 2 ? 1 : 2;
}

mg_status build_faces(int32_t R, HostLevel &L, std::string &err) {
    KeyMap idx;
    idx.reserve(L.keys.size() * 2);
    for (size_t b = 0; b < L.keys.size(); ++b) idx[L.keys[b]] = static_cast<int32_t>(b);
    L.faces.clear();
    L.segs.clear();
    for (size_t b = 0; b < L.keys.size(); ++b) {
        const Key key = L.keys[b];
        int64_t m;
        if (!blocks_per_axis(R, key.lev, m)) {
            err = "block level outside the root grid";
            return MG_ERR_UNBALANCED;
        }
        for (int axis = 0; axis < 3; ++axis) {
            for (int side = 0; side < 2; ++side) {
                int t1, t2;
                tangential(axis, t1, t2);
                Key p = key;
                set_coord(p, axis, coord(key, axis) + (side ? 1 : -1));
                FaceItem fi{};
                fi.blk = static_cast<int32_t>(b);
                fi.nbr = -1;
                fi.axis = static_cast<int8_t>(axis);
                fi.side = static_cast<int8_t>(side);
                if (coord(p, axis) < 0 || coord(p, axis) >= m) {
                    fi.kind = FK_BND;
                    L.faces.push_back(fi);
                    continue;
                }
                auto it = idx.find(p);
                if (it != idx.end()) {
                    fi.kind = FK_SAME;
                    fi.nbr = it->second;
                    L.faces.push_back(fi);
                    continue;
                }
                Key parent{p.p, p.lev - 1, p.i >> 1, p.j >> 1, p.k >> 1};
                it = idx.find(parent);
                if (it != idx.end()) {
                    fi.kind = FK_C2F;
                    fi.nbr = it->second;
                    fi.seg1 = static_cast<int8_t>(coord(key, t1) & 1);
                    fi.seg2 = static_cast<int8_t>(coord(key, t2) & 1);
                    L.faces.push_back(fi);
                    continue;
                }
                for (int s2 = 0; s2 < 2; ++s2) {
                    for (int s1 = 0; s1 < 2; ++s1) {
                        Key c{p.p, p.lev + 1, 0, 0, 0};
                        set_coord(c, axis, 2 * coord(p, axis) + (side == 0 ? 1 : 0));
                        set_coord(c, t1, 2 * coord(p, t1) + s1);
                        set_coord(c, t2, 2 * coord(p, t2) + s2);
                        auto ic = idx.find(c);
                        if (ic == idx.end()) {
                            err = "problem " + std::to_string(key.p) + " leaf (" + std::to_string(key.lev) + "," +
                                  std::to_string(key.i) + "," +
                                  std::to_string(key.j) + "," + std::to_string(key.k) +
                                  ") has a face neighbourhood that is not 2:1 balanced";
                            return MG_ERR_UNBALANCED;
                        }
                        SegItem si{};
                        si.coarse = static_cast<int32_t>(b);
                        si.fine = ic->second;
                        si.axis = static_cast<int8_t>(axis);
                        si.side = static_cast<int8_t>(side);
                        si.s1 = static_cast<int8_t>(s1);
                        si.s2 = static_cast<int8_t>(s2);
                        L.segs.push_back(si);
                    }
                }
            }
        }
    }
    return MG_OK;
}

mg_status validate_leaves(int32_t R, int32_t n_problems, const std::vector<Key> &leaves, std::string &err) {
    if (leaves.empty()) {
        err = "no leaves";
        return MG_ERR_INVALID_ARG;
    }
    KeyMap idx;
    std::vector<int32_t> maxlev(n_problems, 0);
    std::vector<int64_t> count(n_problems, 0);
    for (size_t b = 0; b < leaves.size(); ++b) {
        const Key &k = leaves[b];
        if (k.p < 0 || k.p >= n_problems) {
            err = "leaf problem index outside 0..n_problems-1";
            return MG_ERR_INVALID_ARG;
        }
        int64_t m;
        if (k.lev < 0 || k.lev > 20 || !blocks_per_axis(R, k.lev, m) || k.i < 0 || k.j < 0 || k.k < 0 || k.i >= m ||
            k.j >= m || k.k >= m) {
            err = "leaf outside the domain";
            return MG_ERR_UNBALANCED;
        }
        if (!idx.emplace(k, static_cast<int32_t>(b)).second) {
            err = "duplicate leaf";
            return MG_ERR_UNBALANCED;
        }
        maxlev[k.p] = std::max(maxlev[k.p], k.lev);
        count[k.p] += 1;
    }
    // per problem: no leaf has an ancestor among the leaves, and the volumes (in finest-level units) sum to the
    // domain's
    std::vector<long double> vol(n_problems, 0.0L);
    for (const Key &k : leaves) {
        if ((static_cast<int64_t>(R) << maxlev[k.p]) > (1 << 20)) {
            err = "forest too deep";
            return MG_ERR_INVALID_ARG;
        }
        Key a = k;
        while (a.lev > 0) {
            a = Key{a.p, a.lev - 1, a.i >> 1, a.j >> 1, a.k >> 1};
            if (idx.count(a)) {
                err = "overlapping leaves";
                return MG_ERR_UNBALANCED;
            }
        }
        vol[k.p] += std::ldexp(1.0L, 3 * (maxlev[k.p] - k.lev));
    }
    for (int32_t p = 0; p < n_problems; ++p) {
        const int64_t mfin = static_cast<int64_t>(R) << maxlev[p];
        const long double want = static_cast<long double>(mfin) * mfin * mfin;
        if (count[p] == 0 || vol[p] != want) {
            err = "leaves do not cover the domain (problem " + std::to_string(p) + ")";
            return MG_ERR_UNBALANCED;
        }
    }
    return MG_OK;
}

// For every problem whose level has more than max_coarse unknowns, merge each complete octet of siblings at its
// deepest level into the parent; every other block is carried over.  false if nothing merges.
bool merge_deepest(int32_t R, int32_t n_problems, int64_t max_coarse, const HostLevel &L, HostLevel &C) {
    const int64_t cells = static_cast<int64_t>(L.n) * L.n * L.n;
    std::vector<int32_t> deepest(n_problems, -1000);
    std::vector<int64_t> nblk(n_problems, 0);
    for (const Key &k : L.keys) {
        deepest[k.p] = std::max(deepest[k.p], k.lev);
        nblk[k.p] += 1;
    }
    std::vector<char> wants(n_problems, 0);
    for (int32_t p = 0; p < n_problems; ++p) {
        int64_t m;
        wants[p] = nblk[p] * cells > max_coarse && blocks_per_axis(R, deepest[p] - 1, m);
    }
    KeyMap idx;
    for (size_t b = 0; b < L.keys.size(); ++b) idx[L.keys[b]] = static_cast<int32_t>(b);
    KeyMap counts;
    for (const Key &k : L.keys)
        if (wants[k.p] && k.lev == deepest[k.p]) counts[Key{k.p, k.lev - 1, k.i >> 1, k.j >> 1, k.k >> 1}] += 1;
    std::vector<Key> parents;
    for (auto &kv : counts)
        if (kv.second == 8) parents.push_back(kv.first);
    if (parents.empty()) return false;
    std::sort(parents.begin(), parents.end(), [](const Key &a, const Key &b) {
        if (a.p != b.p) return a.p < b.p;
        if (a.k != b.k) return a.k < b.k;
        if (a.j != b.j) return a.j < b.j;
        return a.i < b.i;
    });
    KeyMap is_parent;
    for (const Key &p : parents) is_parent[p] = 1;
    C.n = L.n;
    C.keys.clear();
    C.to_next.clear();
    std::vector<XferItem> xf;
    for (size_t b = 0; b < L.keys.size(); ++b) {
        const Key &k = L.keys[b];
        if (is_parent.count(Key{k.p, k.lev - 1, k.i >> 1, k.j >> 1, k.k >> 1})) continue;
        C.keys.push_back(k);
        XferItem x{};
        x.kind = XF_COPY;
        x.src[0] = static_cast<int32_t>(b);
        xf.push_back(x);
    }
    for (const Key &p : parents) {
        C.keys.push_back(p);
        XferItem x{};
        x.kind = XF_MERGE;
        for (int o = 0; o < 8; ++o) {
            Key c{p.p, p.lev + 1, 2 * p.i + (o & 1), 2 * p.j + ((o >> 1) & 1), 2 * p.k + ((o >> 2) & 1)};
            x.src[o] = idx.at(c);
        }
        xf.push_back(x);
    }
    C.to_next = xf;  // temporarily holds the transfer from L; moved to L.to_next by the caller
    return true;
}

}  // namespace

void build_diagonal(int32_t R, HostLevel &L) {
    KeyMap idx;
    idx.reserve(L.keys.size() * 2);
    for (size_t b = 0; b < L.keys.size(); ++b) idx[L.keys[b]] = static_cast<int32_t>(b);
    L.edges.clear();
    L.corners.clear();
    // the same-level block at offsets d[0..2] in {-1, 0, 1}, or -1
    const auto across = [&](const Key &key, const int d[3]) -> int32_t {
        int64_t m;
        if (!blocks_per_axis(R, key.lev, m)) return -1;
        Key k2 = key;
        for (int a = 0; a < 3; ++a) {
            const int v = coord(key, a) + d[a];
            if (v < 0 || v >= m) return -1;
            set_coord(k2, a, v);
        }
        const auto it = idx.find(k2);
        return it == idx.end() ? -1 : it->second;
    };
    static const int kPair[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (size_t b = 0; b < L.keys.size(); ++b) {
        const Key key = L.keys[b];
        for (int q = 0; q < 3; ++q)
            for (int bits = 0; bits < 4; ++bits) {
                int d[3] = {0, 0, 0};
                d[kPair[q][0]] = (bits & 1) ? 1 : -1;
                d[kPair[q][1]] = (bits & 2) ? 1 : -1;
                L.edges.push_back({static_cast<int32_t>(b), across(key, d), 4 * q + bits, 0});
            }
        for (int bits = 0; bits < 8; ++bits) {
            const int d[3] = {(bits & 1) ? 1 : -1, (bits & 2) ? 1 : -1, (bits & 4) ? 1 : -1};
            L.corners.push_back({static_cast<int32_t>(b), across(key, d), bits, 0});
        }
    }
}

mg_status build_hierarchy(int32_t R, int32_t n, int32_t n_problems, const std::vector<Key> &leaves,
                          int32_t max_coarse, HostHierarchy &out, std::string &err) {
    if (R < 1 || R > 4096) {
        err = "roots must be in 1..4096";
        return MG_ERR_INVALID_ARG;
    }
    if (n < 4 || (n & (n - 1)) != 0 || n > 1024) {
        err = "n must be a power of two in 4..1024";
        return MG_ERR_BLOCK_SIZE;
    }
    if (n_problems < 1) {
        err = "n_problems must be >= 1";
        return MG_ERR_INVALID_ARG;
    }
    mg_status st = validate_leaves(R, n_problems, leaves, err);
    if (st != MG_OK) return st;
    out.R = R;
    out.levels.clear();
    HostLevel L0;
    L0.n = n;
    L0.keys = leaves;
    out.levels.push_back(L0);
    while (out.levels.back().n > 4) {
        HostLevel nx;
        nx.n = out.levels.back().n / 2;
        nx.keys = out.levels.back().keys;
        std::vector<XferItem> xf(nx.keys.size());
        for (size_t b = 0; b < xf.size(); ++b) {
            xf[b] = XferItem{};
            xf[b].kind = XF_HALVE;
            xf[b].src[0] = static_cast<int32_t>(b);
        }
        out.levels.back().to_next = xf;
        out.levels.push_back(nx);
    }
    for (;;) {
        HostLevel nx;
        if (!merge_deepest(R, n_problems, max_coarse, out.levels.back(), nx)) break;
        out.levels.back().to_next = nx.to_next;
        nx.to_next.clear();
        out.levels.push_back(nx);
    }
    for (HostLevel &L : out.levels) {
        st = build_faces(R, L, err);
        if (st != MG_OK) return st;
        L.h.resize(L.keys.size());
        for (size_t b = 0; b < L.keys.size(); ++b)
            L.h[b] = 1.0 / (static_cast<double>(R) * std::ldexp(1.0, L.keys[b].lev) * L.n);
    }
    return MG_OK;
}

}  // namespace octmg
