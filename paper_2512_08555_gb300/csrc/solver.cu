// Host side of libmrp: forest ingest and validation, device tables, the
// V-cycle schedule (arXiv 2512.08555, Alg. 1) and the C ABI entry points.
#include "mrp_internal.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <unordered_map>

namespace mrp {

static inline uint64_t key3(int x, int y, int z) {
    return ((uint64_t)(uint32_t)x) | ((uint64_t)(uint32_t)y << 21) | ((uint64_t)(uint32_t)z << 42);
}

// ---------------------------------------------------------------- forest
// Host tables of one forest with block indices local to it.
struct OneForest {
    int L = 0;
    std::vector<Level> lv;
    std::vector<int> leaf_block;      // per leaf (caller order): block index at its level
};

static int build_one(const mrp_forest& f, OneForest& out, std::string& why) {
    for (int a = 0; a < 3; ++a)
        if (f.nb0[a] < 1 || f.nb0[a] > 4096) { why = "nb0 out of range"; return MRP_ERR_INVALID_FOREST; }
    if (!(f.h0 > 0.0)) { why = "h0 must be positive"; return MRP_ERR_INVALID_FOREST; }
    if (f.n % 2 != 0 || f.n < 8 || f.n > 24) { why = "block size must be even, 8..24"; return MRP_ERR_INVALID_FOREST; }
    if (f.n_leaves < 1 || !f.leaf_level || !f.leaf_ijk) { why = "no leaves"; return MRP_ERR_INVALID_ARG; }
    int L = 0;
    for (int i = 0; i < f.n_leaves; ++i) {
        const int l = f.leaf_level[i];
        if (l < 0 || l > 20) { why = "leaf level out of range"; return MRP_ERR_INVALID_FOREST; }
        L = std::max(L, l);
        for (int a = 0; a < 3; ++a) {
            const int c = f.leaf_ijk[3 * i + a];
            if (c < 0 || c >= (f.nb0[a] << l)) { why = "leaf outside the domain"; return MRP_ERR_INVALID_FOREST; }
        }
    }
    out.L = L;
    // blocks per level: leaves, then parents of finer blocks
    std::vector<std::unordered_map<uint64_t, int>> idx(L + 1);
    std::vector<std::map<std::array<int, 3>, bool>> all(L + 1);   // (z, y, x) -> is_leaf
    for (int i = 0; i < f.n_leaves; ++i) {
        const int l = f.leaf_level[i];
        const int x = f.leaf_ijk[3 * i], y = f.leaf_ijk[3 * i + 1], z = f.leaf_ijk[3 * i + 2];
        std::array<int, 3> c{z, y, x};
        if (all[l].count(c)) { why = "duplicate leaf"; return MRP_ERR_INVALID_FOREST; }
        all[l][c] = true;
    }
    for (int k = L; k > 0; --k)
        for (auto& kv : all[k]) {
            std::array<int, 3> p{kv.first[0] >> 1, kv.first[1] >> 1, kv.first[2] >> 1};
            auto it = all[k - 1].find(p);
            if (it == all[k - 1].end()) all[k - 1][p] = false;
            else if (it->second) { why = "overlapping leaves"; return MRP_ERR_INVALID_FOREST; }
        }
    out.lv.assign(L + 1, Level());
    for (int k = 0; k <= L; ++k) {
        Level& lv = out.lv[k];
        lv.nb = (int)all[k].size();
        int b = 0;
        for (auto& kv : all[k]) {   // std::map order: z, then y, then x
            const int z = kv.first[0], y = kv.first[1], x = kv.first[2];
            lv.h_coords.push_back(x); lv.h_coords.push_back(y); lv.h_coords.push_back(z);
            lv.h_is_leaf.push_back(kv.second ? 1 : 0);
            idx[k][key3(x, y, z)] = b++;
        }
    }
    if (out.lv[0].nb != f.nb0[0] * f.nb0[1] * f.nb0[2]) { why = "leaves do not tile the domain"; return MRP_ERR_INVALID_FOREST; }
    auto find = [&](int k, int x, int y, int z) -> int {
        if (x < 0 || y < 0 || z < 0 || x >= (f.nb0[0] << k) || y >= (f.nb0[1] << k) || z >= (f.nb0[2] << k)) return NBR_OUTSIDE;
        auto it = idx[k].find(key3(x, y, z));
        return it == idx[k].end() ? NBR_MISSING : it->second;
    };
    for (int k = 0; k <= L; ++k) {
        Level& lv = out.lv[k];
        lv.h_nbr.resize((size_t)lv.nb * 27);
        lv.h_parent.assign(lv.nb, -1);
        lv.h_octant.assign(lv.nb, 0);
        lv.h_children.assign((size_t)lv.nb * 8, -1);
        for (int b = 0; b < lv.nb; ++b) {
            const int x = lv.h_coords[3 * b], y = lv.h_coords[3 * b + 1], z = lv.h_coords[3 * b + 2];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        lv.h_nbr[(size_t)27 * b + dir27(dx, dy, dz)] = find(k, x + dx, y + dy, z + dz);
            if (k > 0) {
                lv.h_parent[b] = find(k - 1, x >> 1, y >> 1, z >> 1);
                lv.h_octant[b] = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
            }
            if (lv.h_is_leaf[b]) continue;
            for (int o = 0; o < 8; ++o) {
                const int c = k < L ? find(k + 1, 2 * x + (o & 1), 2 * y + ((o >> 1) & 1), 2 * z + ((o >> 2) & 1)) : -1;
                if (c < 0) { why = "leaves do not tile the domain"; return MRP_ERR_INVALID_FOREST; }
                lv.h_children[(size_t)8 * b + o] = c;
            }
            if (k == 0 && (x == 0 || y == 0 || z == 0 || x == f.nb0[0] - 1 || y == f.nb0[1] - 1 || z == f.nb0[2] - 1)) {
                why = "a block touching the unbounded boundary is refined";
                return MRP_ERR_INVALID_FOREST;
            }
        }
    }
    // 2:1 balance across faces, edges and corners: each of the 26 neighbour
    // positions of a level-k block lies in a block of level k-1.
    for (int k = 1; k <= L; ++k) {
        const Level& lv = out.lv[k];
        for (int b = 0; b < lv.nb; ++b) {
            const int x = lv.h_coords[3 * b], y = lv.h_coords[3 * b + 1], z = lv.h_coords[3 * b + 2];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int qx = x + dx, qy = y + dy, qz = z + dz;
                        if (qx < 0 || qy < 0 || qz < 0) { why = "2:1 balance violated"; return MRP_ERR_INVALID_FOREST; }
                        if (find(k - 1, qx >> 1, qy >> 1, qz >> 1) < 0) { why = "2:1 balance violated"; return MRP_ERR_INVALID_FOREST; }
                    }
        }
    }
    out.leaf_block.resize(f.n_leaves);
    for (int i = 0; i < f.n_leaves; ++i)
        out.leaf_block[i] = find(f.leaf_level[i], f.leaf_ijk[3 * i], f.leaf_ijk[3 * i + 1], f.leaf_ijk[3 * i + 2]);
    return MRP_OK;
}

// Pools the problems' blocks per level (problem after problem), with the
// neighbour, parent and child tables re-indexed into the pools.
int build_forest(Handle& h, const std::vector<ProblemDesc>& list, std::string& why) {
    if (list.empty()) { why = "no problems"; return MRP_ERR_INVALID_ARG; }
    h.n = list[0].f->n;
    h.h0 = list[0].f->h0;
    std::vector<OneForest> one(list.size());
    int L = 0;
    for (size_t p = 0; p < list.size(); ++p) {
        if (list[p].f->n != h.n) { why = "problems of one handle share the block size"; return MRP_ERR_INVALID_ARG; }
        const int rc = build_one(*list[p].f, one[p], why);
        if (rc) return rc;
        L = std::max(L, one[p].L);
    }
    h.L = L;
    h.lv.assign(L + 1, Level());
    h.pr.assign(list.size(), Problem());
    std::vector<std::vector<int>> base(list.size(), std::vector<int>(L + 2, 0));
    for (int k = 0; k <= L; ++k) {
        int b = 0;
        for (size_t p = 0; p < list.size(); ++p) {
            base[p][k] = b;
            if (k <= one[p].L) b += one[p].lv[k].nb;
        }
        h.lv[k].nb = b;
    }
    for (size_t p = 0; p < list.size(); ++p) {
        const mrp_forest& f = *list[p].f;
        Problem& pr = h.pr[p];
        pr.forest = list[p].forest;
        pr.comp = list[p].comp;
        pr.h0 = f.h0;
        pr.scale = (f.h0 / h.h0) * (f.h0 / h.h0);
        pr.L = one[p].L;
        pr.base0 = base[p][0];
        for (int a = 0; a < 3; ++a) { pr.nb0[a] = f.nb0[a]; pr.n0[a] = f.nb0[a] * f.n; }
        for (int k = 0; k <= one[p].L; ++k) {
            const Level& s = one[p].lv[k];
            Level& d = h.lv[k];
            const int off = base[p][k];
            const int offc = k > 0 ? base[p][k - 1] : 0, offf = base[p][k + 1];
            d.h_coords.insert(d.h_coords.end(), s.h_coords.begin(), s.h_coords.end());
            d.h_is_leaf.insert(d.h_is_leaf.end(), s.h_is_leaf.begin(), s.h_is_leaf.end());
            d.h_octant.insert(d.h_octant.end(), s.h_octant.begin(), s.h_octant.end());
            for (int v : s.h_nbr) d.h_nbr.push_back(v >= 0 ? v + off : v);
            for (int v : s.h_parent) d.h_parent.push_back(v >= 0 ? v + offc : v);
            for (int v : s.h_children) d.h_children.push_back(v >= 0 ? v + offf : v);
            for (int b = 0; b < s.nb; ++b) d.h_prob.push_back((int)p);
        }
    }
    for (int k = 0; k <= L; ++k) {
        Level& lv = h.lv[k];
        for (int b = 0; b < lv.nb; ++b) (lv.h_is_leaf[b] ? lv.h_leaf_blocks : lv.h_cov_blocks).push_back(b);
        lv.nleaf = (int)lv.h_leaf_blocks.size();
        lv.ncov = (int)lv.h_cov_blocks.size();
        // launch order: blocks that interpolate ghosts (heavier) first
        auto interp = [&](int b) {
            for (int d = 0; d < 27; ++d) if (lv.h_nbr[(size_t)27 * b + d] == NBR_MISSING) return true;
            return false;
        };
        for (int pass = 0; pass < 2; ++pass)
            for (int b = 0; b < lv.nb; ++b) if (interp(b) == (pass == 0)) lv.h_order.push_back(b);
        lv.nint = 0;
        for (int b = 0; b < lv.nb; ++b) lv.nint += interp(b) ? 1 : 0;
        std::stable_partition(lv.h_leaf_blocks.begin(), lv.h_leaf_blocks.end(), interp);
    }
    // level-0 list ranges per problem (level 0 never interpolates, so its lists stay in block order)
    const Level& l0 = h.lv[0];
    for (size_t p = 0; p < list.size(); ++p) {
        Problem& pr = h.pr[p];
        const int lo = pr.base0, hi = pr.base0 + pr.nb0[0] * pr.nb0[1] * pr.nb0[2];
        auto range = [&](const std::vector<int>& v, int& a, int& b) {
            a = (int)(std::lower_bound(v.begin(), v.end(), lo) - v.begin());
            b = (int)(std::lower_bound(v.begin(), v.end(), hi) - v.begin());
        };
        range(l0.h_leaf_blocks, pr.leaf0_lo, pr.leaf0_hi);
        range(l0.h_cov_blocks, pr.cov0_lo, pr.cov0_hi);
    }
    // leaves in the caller's order, with their element offsets and scales
    h.n_leaves = 0;
    h.h_leaf_level.clear(); h.h_leaf_block.clear(); h.h_leaf_src.clear(); h.h_leaf_scale.clear();
    const int64_t n3 = (int64_t)h.n * h.n * h.n;
    for (size_t p = 0; p < list.size(); ++p) {
        const mrp_forest& f = *list[p].f;
        for (int i = 0; i < f.n_leaves; ++i) {
            const int l = f.leaf_level[i];
            h.h_leaf_level.push_back(l);
            h.h_leaf_block.push_back(one[p].leaf_block[i] + base[p][l]);
            h.h_leaf_src.push_back(list[p].src_off + (int64_t)i * n3);
            h.h_leaf_scale.push_back(h.pr[p].scale);
        }
        h.n_leaves += f.n_leaves;
    }
    h.leaf_nodes = (int64_t)h.n_leaves * n3;
    h.total_nodes = 0;
    for (int k = 0; k <= L; ++k) h.total_nodes += (int64_t)h.lv[k].nb * n3;
    h.fstar.assign(list.size(), 0.0);
    return MRP_OK;
}

template <typename T>
static int up(T*& d, const std::vector<T>& v) {
    if (v.empty()) { d = nullptr; return MRP_OK; }
    if (cudaMalloc(&d, sizeof(T) * v.size()) != cudaSuccess) return MRP_ERR_OOM;
    if (cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) return MRP_ERR_CUDA;
    return MRP_OK;
}

static int alloc_field(double*& p, size_t count) {
    if (count == 0) { p = nullptr; return MRP_OK; }
    if (cudaMalloc(&p, sizeof(double) * count) != cudaSuccess) return MRP_ERR_OOM;
    if (cudaMemset(p, 0, sizeof(double) * count) != cudaSuccess) return MRP_ERR_CUDA;
    return MRP_OK;
}

// Neighbourhood records of every block (layout: REC_* in mrp_internal.h).
// The interpolated regions are the directions without a same-level
// neighbour; each takes TN^2 (face), TN (edge) or 1 (corner) entries of the
// normal-reduced array and, for faces, n TN entries of the face array.  The
// coarse patch (indices 0..PL-1 per axis, PL = n/2 + I) is needed on
// [0, I) for a -1 side, at index `up` (the coarse node of fine coordinate n)
// for a +1 side and on [1, PL) along a tangential axis.
static void build_records(Handle& h) {
    const int n = h.n, I = h.M + 2, hh = n / 2;
    const int TN = hh + I - 1, PL = hh + I, plo = 4 - I / 2, up = 4 + hh - plo;
    for (size_t k = 0; k < h.lv.size(); ++k) {
        Level& lv = h.lv[k];
        lv.h_rec.assign((size_t)lv.nb * REC_INTS, 0);
        for (int b = 0; b < lv.nb; ++b) {
            int* r = &lv.h_rec[(size_t)b * REC_INTS];
            for (int d = 0; d < 27; ++d) r[REC_SNBR + d] = lv.h_nbr[(size_t)27 * b + d];
            for (int d = 0; d < 27; ++d) {
                int cb = NBR_OUTSIDE;
                if (k > 0 && lv.h_parent[b] >= 0) cb = h.lv[k - 1].h_nbr[(size_t)27 * lv.h_parent[b] + d];
                r[REC_PNBR + d] = cb;
                const bool inner = cb >= 0 && !h.lv[k - 1].h_is_leaf[cb];
                for (int o = 0; o < 8; ++o)
                    r[REC_PCH + 8 * d + o] = inner ? h.lv[k - 1].h_children[(size_t)8 * cb + o] : -1;
            }
            int o = 0, oa = 0, oc = 0, od = 0, nr = 0;
            int lo[3] = {PL, PL, PL}, hi[3] = {0, 0, 0};
            for (int d = 0; d < 27; ++d) {
                if (d == 13 || r[REC_SNBR + d] != NBR_MISSING) continue;
                const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
                int nt = 0;
                for (int a = 0; a < 3; ++a) {
                    const int l = dd[a] < 0 ? 0 : (dd[a] > 0 ? up : 1);
                    const int e = dd[a] < 0 ? I : (dd[a] > 0 ? up + 1 : PL);
                    nt += dd[a] == 0;
                    lo[a] = std::min(lo[a], l);
                    hi[a] = std::max(hi[a], e);
                }
                r[REC_RDIR + nr] = d;
                r[REC_ROFF + nr] = o;
                r[REC_RAOFF + nr] = oa;
                r[REC_COFF + nr] = oc;
                r[REC_DOFF + nr] = od;
                o += nt == 2 ? TN * TN : (nt == 1 ? TN : 1);
                oa += nt == 2 ? n * TN : 0;
                oc += nt == 2 ? n * TN : (nt == 1 ? n : 1);
                od += nt == 2 ? n * n : 0;
                ++nr;
            }
            r[REC_NREG] = nr;
            r[REC_NTOT] = o;
            r[REC_NTOT + 1] = oc;
            r[REC_NTOT + 2] = od;
            for (int a = 0; a < 3; ++a) { r[REC_LO + a] = nr ? lo[a] : 0; r[REC_HI + a] = nr ? hi[a] : 0; }
        }
    }
}

int upload_tables(Handle& h) {
    int rc;
    build_records(h);
    const size_t n = h.n, S = n + 2, S4 = n + 4;
    for (Level& lv : h.lv) {
        if ((rc = up(lv.coords, lv.h_coords))) return rc;
        if ((rc = up(lv.nbr, lv.h_nbr))) return rc;
        if ((rc = up(lv.parent, lv.h_parent))) return rc;
        if ((rc = up(lv.octant, lv.h_octant))) return rc;
        if ((rc = up(lv.children, lv.h_children))) return rc;
        if ((rc = up(lv.leaf_blocks, lv.h_leaf_blocks))) return rc;
        if ((rc = up(lv.cov_blocks, lv.h_cov_blocks))) return rc;
        if ((rc = up(lv.order, lv.h_order))) return rc;
        if ((rc = up(lv.is_leaf, lv.h_is_leaf))) return rc;
        if ((rc = up(lv.prob, lv.h_prob))) return rc;
        if ((rc = up(lv.rec, lv.h_rec))) return rc;
        if ((rc = alloc_field(lv.U, lv.nb * S * S * S))) return rc;
        if ((rc = alloc_field(lv.Ualt, lv.nb * S * S * S))) return rc;
        if ((rc = alloc_field(lv.F, lv.nb * n * n * n))) return rc;
        if ((rc = alloc_field(lv.R, lv.nb * n * n * n))) return rc;
        if ((rc = alloc_field(lv.H, lv.nb * n * n * n))) return rc;
        if (h.M == 6 && (rc = alloc_field(lv.Fraw, lv.nb * S4 * S4 * S4))) return rc;   // R^6: two ghost layers
        if (h.stop_rule == MRP_STOP_CAUCHY && (rc = alloc_field(lv.Uprev, lv.nb * n * n * n))) return rc;
    }
    if ((rc = up(h.leaf_level, h.h_leaf_level))) return rc;
    if ((rc = up(h.leaf_block, h.h_leaf_block))) return rc;
    if ((rc = up(h.leaf_src, h.h_leaf_src))) return rc;
    if ((rc = up(h.leaf_scale, h.h_leaf_scale))) return rc;
    const size_t nslot = 4 * h.pr.size();
    if (cudaMalloc(&h.dmax, sizeof(unsigned long long) * nslot) != cudaSuccess) return MRP_ERR_OOM;
    if (cudaMallocHost(&h.hmax, sizeof(unsigned long long) * nslot) != cudaSuccess) return MRP_ERR_OOM;
    return MRP_OK;
}

static void release(Handle& h) {
    adjoint_release(h);
    for (Level& lv : h.lv) {
        cudaFree(lv.coords); cudaFree(lv.nbr); cudaFree(lv.parent); cudaFree(lv.octant); cudaFree(lv.children);
        cudaFree(lv.leaf_blocks); cudaFree(lv.cov_blocks); cudaFree(lv.is_leaf); cudaFree(lv.order); cudaFree(lv.prob);
        cudaFree(lv.rec);
        cudaFree(lv.U); cudaFree(lv.F); cudaFree(lv.R); cudaFree(lv.H); cudaFree(lv.Fraw);
        cudaFree(lv.U32); cudaFree(lv.F32); cudaFree(lv.R32); cudaFree(lv.H32);
        cudaFree(lv.Ualt); cudaFree(lv.U32alt); cudaFree(lv.Uprev);
    }
    h.lv.clear();
    for (Problem& p : h.pr) {
        for (int a = 0; a < 3; ++a) { cudaFree(p.ax[a].tw); cudaFree(p.ax[a].tw32); }
        cudaFree(p.ghat); cudaFree(p.ghat32);
    }
    h.pr.clear();
    cudaFree(h.spec32); cudaFree(h.c0); cudaFree(h.off32);
    cudaFree(h.leaf_level); cudaFree(h.leaf_block); cudaFree(h.leaf_src); cudaFree(h.leaf_scale);
    cudaFree(h.spec); cudaFree(h.lgf); cudaFree(h.dmax);
    if (h.hmax) cudaFreeHost(h.hmax);
    h.hmax = nullptr;
    for (cudaEvent_t e : h.ev) cudaEventDestroy(e);
    h.ev.clear();
}

// FP32 workspace of the mixed-precision path: per-level fields, FP32 copies
// of the twiddles and of the Green's-function spectrum, the FP32 spectral
// buffer, and the level-0 injection mismatch (FP64) with its FP32 offset.
static int mixed_setup(Handle& h) {
    const size_t n = h.n, S = n + 2;
    for (Level& lv : h.lv) {
        const size_t nb = lv.nb;
        if (cudaMalloc(&lv.U32, sizeof(float) * nb * S * S * S) != cudaSuccess) return MRP_ERR_OOM;
        if (cudaMalloc(&lv.U32alt, sizeof(float) * nb * S * S * S) != cudaSuccess) return MRP_ERR_OOM;
        cudaMemset(lv.U32alt, 0, sizeof(float) * nb * S * S * S);
        if (cudaMalloc(&lv.F32, sizeof(float) * nb * n * n * n) != cudaSuccess) return MRP_ERR_OOM;
        if (cudaMalloc(&lv.R32, sizeof(float) * nb * n * n * n) != cudaSuccess) return MRP_ERR_OOM;
        if (cudaMalloc(&lv.H32, sizeof(float) * nb * n * n * n) != cudaSuccess) return MRP_ERR_OOM;
        cudaMemset(lv.U32, 0, sizeof(float) * nb * S * S * S);
        cudaMemset(lv.F32, 0, sizeof(float) * nb * n * n * n);
        cudaMemset(lv.R32, 0, sizeof(float) * nb * n * n * n);
        cudaMemset(lv.H32, 0, sizeof(float) * nb * n * n * n);
    }
    const size_t nb0 = h.lv[0].nb;
    if (cudaMalloc(&h.c0, sizeof(double) * nb0 * n * n * n) != cudaSuccess) return MRP_ERR_OOM;
    if (cudaMalloc(&h.off32, sizeof(float) * nb0 * n * n * n) != cudaSuccess) return MRP_ERR_OOM;
    cudaMemset(h.c0, 0, sizeof(double) * nb0 * n * n * n);
    cudaMemset(h.off32, 0, sizeof(float) * nb0 * n * n * n);
    size_t ns = 0;
    for (Problem& p : h.pr) {
        for (int a = 0; a < 3; ++a) {
            const int P = p.ax[a].P;
            std::vector<double2> tw(P);
            std::vector<float2> tw32(P);
            if (cudaMemcpy(tw.data(), p.ax[a].tw, sizeof(double2) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
                return MRP_ERR_CUDA;
            for (int m = 0; m < P; ++m) tw32[m] = make_float2((float)tw[m].x, (float)tw[m].y);
            if (cudaMalloc(&p.ax[a].tw32, sizeof(float2) * P) != cudaSuccess) return MRP_ERR_OOM;
            if (cudaMemcpy(p.ax[a].tw32, tw32.data(), sizeof(float2) * P, cudaMemcpyHostToDevice) != cudaSuccess)
                return MRP_ERR_CUDA;
        }
        const size_t ng = (size_t)p.gK[0] * p.gK[1] * p.gK[2];
        std::vector<double> g(ng);
        std::vector<float> g32(ng);
        if (cudaMemcpy(g.data(), p.ghat, sizeof(double) * ng, cudaMemcpyDeviceToHost) != cudaSuccess) return MRP_ERR_CUDA;
        for (size_t i = 0; i < ng; ++i) g32[i] = (float)g[i];
        if (cudaMalloc(&p.ghat32, sizeof(float) * ng) != cudaSuccess) return MRP_ERR_OOM;
        if (cudaMemcpy(p.ghat32, g32.data(), sizeof(float) * ng, cudaMemcpyHostToDevice) != cudaSuccess) return MRP_ERR_CUDA;
        ns = std::max(ns, (size_t)p.ax[2].P * p.ax[1].P * p.ax[0].K);
    }
    if (cudaMalloc(&h.spec32, sizeof(float2) * ns) != cudaSuccess) return MRP_ERR_OOM;
    return MRP_OK;
}

// ---------------------------------------------------------------- schedule (Alg. 1)
void harvest(Handle& h) {
    for (const auto& p : h.pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h.ev[p.e0], h.ev[p.e0 + 1]) == cudaSuccess) {
            h.prof_ms[p.phase] += ms;
            h.prof_cnt[p.phase] += 1;
            h.prof_nodes[p.phase] += p.nodes;
        }
    }
    h.pend.clear();
    h.ev_used = 0;
}

static int64_t halo_nodes(const Handle& h, int g) { const int64_t S = h.n + 2 * g; return S * S * S - n3(h); }

// Per-level fields of one working precision: FP64 (plain path and outer
// refinement) or FP32 (inner cycles of the mixed path).
template <typename T> struct Fld { T *U, *F, *R, *H; };
template <typename T> static Fld<T> fld(Handle& h, int k) {
    if constexpr (sizeof(T) == 8) return Fld<T>{h.lv[k].U, h.lv[k].F, h.lv[k].R, h.lv[k].H};
    else return Fld<T>{h.lv[k].U32, h.lv[k].F32, h.lv[k].R32, h.lv[k].H32};
}
// Offset added when level 1 is restricted into the covered level-0 nodes: the
// FP32 correction cycles carry -c0 in the level-0 state there (see
// kernels_mixed.cu); ghost interpolation of level 1 reads the plain injection.
template <typename T> static const T* off0(Handle& h) {
    if constexpr (sizeof(T) == 4) return h.mixed ? h.off32 : nullptr;
    else return nullptr;
}

template <typename T> static T*& ualt(Handle& h, int k) {
    if constexpr (sizeof(T) == 8) return h.lv[k].Ualt;
    else return h.lv[k].U32alt;
}
template <typename T> static T*& ucur(Handle& h, int k) {
    if constexpr (sizeof(T) == 8) return h.lv[k].U;
    else return h.lv[k].U32;
}
template <typename T> static const T* ucoarse(Handle& h, int k) { return k >= 1 ? ucur<T>(h, k - 1) : nullptr; }

// Covered level-(k-1) nodes take the injection of the level-k values.
template <typename T>
static void inject_level(Handle& h, int k, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_GHOST), h.lv[k].nb * n3(h) / 8, 1);
    launch_inject_to_parent<T>(ucur<T>(h, k - 1), 1, ucur<T>(h, k), 1, h.lv[k].view(), h.n, nullptr, s);
}

// Ghosting of u on level k into the stored ghost layer (step API): the
// injection into the covered level-(k-1) nodes, then the ghost layer that the
// fused kernels build in shared memory.
template <typename T>
static void ghost_u(Handle& h, int k, cudaStream_t s) {
    if (k >= 1) inject_level<T>(h, k, s);
    PhaseScope ps(h, s, ph<T>(PH_GHOST), h.lv[k].nb * halo_nodes(h, 1), 1);
    launch_halo_dump<T>(ucur<T>(h, k), ucoarse<T>(h, k), h.lv[k].view(), view_or_empty(h, k - 1), h.n, h.M, s);
}

template <typename T> static constexpr int pidx() { return sizeof(T) == 4 ? 1 : 0; }
// Launches of a fused stencil kernel on a level.
static int fused_launches(const Level& lv) { return lv.nb > 0 ? 1 : 0; }

// One Gauss-Seidel sweep with its ghost layer built in the kernel; reads the
// current buffer, writes the other, then the two swap.
template <typename T>
static void smooth(Handle& h, int k, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_SMOOTH), h.lv[k].nb * n3(h), fused_launches(h.lv[k]));
    const double hk = level_h(h, k);
    launch_smooth_fused<T>(ualt<T>(h, k), ucur<T>(h, k), fld<T>(h, k).F, ucoarse<T>(h, k), h.lv[k].view(),
                           view_or_empty(h, k - 1), h.n, h.M, hk * hk, h.nt_smooth[pidx<T>()][k], s);
    std::swap(ualt<T>(h, k), ucur<T>(h, k));
}

template <typename T>
static void residual(Handle& h, int k, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_RESIDUAL), h.lv[k].nb * n3(h), fused_launches(h.lv[k]));
    const double hk = level_h(h, k);
    launch_residual_fused<T>(fld<T>(h, k).R, ucur<T>(h, k), fld<T>(h, k).F, ucoarse<T>(h, k), h.lv[k].view(),
                             view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), h.nt_res[pidx<T>()][k], s);
}

// Restriction k -> k-1: inject u, full-weight r, FAS RHS on covered blocks, u-hat.
template <typename T>
static void restrict_level(Handle& h, int k, cudaStream_t s) {
    Level& c = h.lv[k - 1];
    {
        PhaseScope ps(h, s, ph<T>(PH_RESTRICT), c.ncov * n3(h), h.lv[k].nb > 0 ? 1 : 0);
        launch_restrict<T>(ucur<T>(h, k - 1), fld<T>(h, k - 1).F, ucur<T>(h, k), fld<T>(h, k).R, h.lv[k].view(), h.n,
                           k == 1 ? off0<T>(h) : nullptr, s);
    }
    PhaseScope ps(h, s, ph<T>(PH_RESTRICT), c.nb * n3(h), fused_launches(c));
    const double hk = level_h(h, k - 1);
    launch_fas_fused<T>(fld<T>(h, k - 1).F, fld<T>(h, k - 1).H, ucur<T>(h, k - 1), ucoarse<T>(h, k - 1), c.view(),
                        view_or_empty(h, k - 2), h.n, h.M, 1.0 / (hk * hk), h.nt_fas[pidx<T>()][k - 1], s);
}

template <typename T>
static void coarse_solve(Handle& h, cudaStream_t s) {
    int64_t nodes = 0;
    for (const Problem& p : h.pr) nodes += (int64_t)p.n0[0] * p.n0[1] * p.n0[2];
    PhaseScope ps(h, s, ph<T>(PH_COARSE), nodes, 5 * h.nprob());
    launch_coarse_solve_t<T>(h, fld<T>(h, 0).F, ucur<T>(h, 0), s);
}

template <typename T>
static void prolong(Handle& h, int k, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_PROLONG), h.lv[k].nb * n3(h), 1);
    launch_prolong<T>(ucur<T>(h, k), ucur<T>(h, k - 1), fld<T>(h, k - 1).H, h.lv[k].view(), h.lv[k - 1].view(), h.n, s);
}

static void prepare_rhs(Handle& h, const double* f, cudaStream_t s) {
    if (h.M <= 4) {
        // R^2, R^4 read one ghost layer: raw f goes into the FP64 u arrays
        // (zero ghost layers; u is cleared again before the cycles), covered
        // nodes take its injection, and each level's f* is formed with its
        // ghost layer built in the kernel, which also takes max |f*| (slot 0)
        PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, 1 + h.L + (h.L + 1));
        const size_t S = h.n + 2;
        LevelPtrs lp{};
        for (int k = 0; k <= h.L; ++k) {
            cudaMemsetAsync(h.lv[k].U, 0, sizeof(double) * h.lv[k].nb * S * S * S, s);
            lp.p[k] = h.lv[k].U;
        }
        launch_scatter_leaves_to(h, f, lp, 1, true, s);
        for (int k = h.L - 1; k >= 0; --k)
            launch_inject_to_parent<double>(h.lv[k].U, 1, h.lv[k + 1].U, 1, h.lv[k + 1].view(), h.n, nullptr, s);
        for (int k = 0; k <= h.L; ++k)
            launch_rhs_fused(h.lv[k].F, h.lv[k].U, k >= 1 ? h.lv[k - 1].U : nullptr, h.lv[k].leaf_blocks, h.lv[k].nleaf,
                             h.lv[k].view(), h.n, h.M, h.slot(0), s);
        return;
    }
    PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, 1 + h.L + 2 * (h.L + 1));
    const size_t S4 = h.n + 4;
    for (int k = 0; k <= h.L; ++k) cudaMemsetAsync(h.lv[k].Fraw, 0, sizeof(double) * h.lv[k].nb * S4 * S4 * S4, s);
    launch_scatter_leaves(h, f, s);
    for (int k = h.L - 1; k >= 0; --k)
        launch_inject_to_parent<double>(h.lv[k].Fraw, 2, h.lv[k + 1].Fraw, 2, h.lv[k + 1].view(), h.n, nullptr, s);
    for (int k = 0; k <= h.L; ++k)
        launch_ghost_fill(h.lv[k].Fraw, 2, k >= 1 ? h.lv[k - 1].Fraw : nullptr, 2, h.lv[k].view(), view_or_empty(h, k - 1),
                          h.n, h.M, true, s);
    for (int k = 0; k <= h.L; ++k) launch_rhs_star(h.lv[k].F, h.lv[k].Fraw, h.lv[k].leaf_blocks, h.lv[k].nleaf, h.n, h.M, s);
}

// One adaptive V(nu1, nu2) cycle, Alg. 1, in precision T.
template <typename T>
void vcycle(Handle& h, cudaStream_t s) {
    for (int k = h.L; k >= 1; --k) {
        for (int i = 0; i < h.nu1; ++i) smooth<T>(h, k, s);
        residual<T>(h, k, s);
        restrict_level<T>(h, k, s);
    }
    coarse_solve<T>(h, s);
    for (int k = 1; k <= h.L; ++k) {
        prolong<T>(h, k, s);
        for (int i = 0; i < h.nu2; ++i) smooth<T>(h, k, s);
    }
}

template void vcycle<double>(Handle&, cudaStream_t);
template void vcycle<float>(Handle&, cudaStream_t);

static double as_double(unsigned long long b) { double d; std::memcpy(&d, &b, sizeof d); return d; }

int read_max(Handle& h, cudaStream_t s, double* out, int slot) {
    const int np = h.nprob();
    if (cudaMemcpyAsync(h.hmax + (size_t)slot * np, h.slot(slot), sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
        return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    for (int p = 0; p < np; ++p) out[p] = as_double(h.hmax[(size_t)slot * np + p]);
    harvest(h);
    return MRP_OK;
}

// ---------------------------------------------------------------- solve, in steps
// A solve is begin (right-hand side, its norms), then step / check pairs until
// every problem of the handle meets the stop rule, then end (the leaf
// values).  Steps only launch work on the stream; checks synchronise it.  A
// handle with several block sizes runs one such sequence per block size, in
// lockstep, each on its own stream.
struct SolveState {
    // per problem: max |f*| (or 1), the last value of the stop rule and the
    // last relative residual (equal to rel under the residual rule)
    std::vector<double> scale, rel, res;
    int cycles = 0, ir = 0;
    bool started = false, done = false;
    int rc = MRP_OK;
    double worst() const {
        double w = 0.0;
        for (double r : rel) w = std::max(w, r);
        return w;
    }
    double worst_res() const {
        double w = 0.0;
        for (double r : res) w = std::max(w, r);
        return w;
    }
};

// CTA size of each fused stencil kernel, per precision and level: the fastest
// of 128, 256 and 512 threads on the level's own block pool (few blocks
// favour large CTAs, which shorten the serial colour sweeps of one block;
// many blocks favour smaller ones).  The timed launches write only scratch
// that every solve overwrites before reading (the other ping-pong buffer, R,
// and F, H of covered blocks).
template <typename T>
static void tune_precision(Handle& h, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    const std::vector<int> cta = {128, 256, 512};
    // the smoother (and the FP32 residual) may also read the right-hand side
    // from global memory
    std::vector<int> smooth_cand = cta;
    for (int c : {128, 256}) smooth_cand.push_back(c | SMOOTH_NOSTAGE);
    constexpr int pi = pidx<T>();
    auto pick_from = [&](const std::vector<int>& cand, auto&& launch) {
        float best = 1e30f;
        int arg = 256;
        for (int c : cand) {
            launch(c);
            for (int rep = 0; rep < 2; ++rep) {      // the faster of two timings of 3 launches
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) launch(c);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) { best = ms; arg = c; }
            }
        }
        return arg;
    };
    auto pick = [&](auto&& launch) { return pick_from(cta, launch); };
    for (int k = 0; k <= h.L; ++k) {
        const double hk = level_h(h, k);
        Level& lv = h.lv[k];
        if (k >= 1) {
            h.nt_smooth[pi][k] = pick_from(smooth_cand, [&](int nt) {
                launch_smooth_fused<T>(ualt<T>(h, k), ucur<T>(h, k), fld<T>(h, k).F, ucoarse<T>(h, k), lv.view(),
                                       view_or_empty(h, k - 1), h.n, h.M, hk * hk, nt, s);
            });
            h.nt_res[pi][k] = pick_from(sizeof(T) == 4 ? smooth_cand : cta, [&](int nt) {
                launch_residual_fused<T>(fld<T>(h, k).R, ucur<T>(h, k), fld<T>(h, k).F, ucoarse<T>(h, k), lv.view(),
                                         view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), nt, s);
            });
        }
        if (k < h.L)
            h.nt_fas[pi][k] = pick([&](int nt) {
                launch_fas_fused<T>(fld<T>(h, k).F, fld<T>(h, k).H, ucur<T>(h, k), ucoarse<T>(h, k), lv.view(),
                                    view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), nt, s);
            });
        if (pi == 0 && lv.nleaf > 0)
            h.nt_leafres[k] = pick([&](int nt) {
                launch_leafres_fused(nullptr, lv.U, lv.F, ucoarse<double>(h, k), lv.leaf_blocks, lv.nleaf, lv.view(),
                                     view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), h.slot(3), nt, s);
            });
    }
}

static void tune_defaults(Handle& h) {
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < Handle::MAXL; ++k) {
            h.nt_smooth[p][k] = h.nt_res[p][k] = h.nt_fas[p][k] = 256;
            h.nt_leafres[k] = 256;
        }
}

int autotune(Handle& h, cudaStream_t s) {
    if (h.tuned) return MRP_OK;
    tune_defaults(h);
    if (h.launch_override) {
        // the NOSTAGE flag applies to the kernels that stage a right-hand side
        const int ct = h.launch_override & ~MRP_LAUNCH_NOSTAGE;
        const int cs = (h.launch_override & MRP_LAUNCH_NOSTAGE) ? (ct | SMOOTH_NOSTAGE) : ct;
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < Handle::MAXL; ++k) {
                h.nt_smooth[p][k] = h.nt_res[p][k] = cs;
                h.nt_fas[p][k] = ct;
                h.nt_leafres[k] = ct;
            }
        h.tuned = true;
        return MRP_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MRP_ERR_CUDA; }
    tune_precision<double>(h, s, e0, e1);
    if (h.mixed) tune_precision<float>(h, s, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    h.tuned = true;
    return MRP_OK;
}

void solve_begin(Handle& h, const double* f, cudaStream_t s) {
    const size_t S = h.n + 2;
    if (h.mixed) cudaMemsetAsync(h.lv[0].F, 0, sizeof(double) * h.lv[0].nb * n3(h), s);
    // max |f*| over the leaves (slot 0): taken while f* is formed for M = 2, 4
    cudaMemsetAsync(h.slot(0), 0, sizeof(unsigned long long) * h.nprob(), s);
    prepare_rhs(h, f, s);
    if (h.M > 4) {
        PhaseScope ps(h, s, PH_NORM, h.leaf_nodes, h.L + 1);
        for (int k = 0; k <= h.L; ++k)
            launch_absmax(h.lv[k].F, h.lv[k].leaf_blocks, h.lv[k].nleaf, h.n, h.slot(0), h.lv[k].prob, s);
    }
    for (int k = 0; k <= h.L; ++k) cudaMemsetAsync(h.lv[k].U, 0, sizeof(double) * h.lv[k].nb * S * S * S, s);
    if (h.stop_rule == MRP_STOP_CAUCHY)          // the iterate before the first cycle: u = 0
        for (int k = 0; k <= h.L; ++k) cudaMemsetAsync(h.lv[k].Uprev, 0, sizeof(double) * h.lv[k].nb * n3(h), s);
}

static int solve_begin_read(Handle& h, cudaStream_t s, SolveState& st) {
    const int rc = read_max(h, s, h.fstar.data(), 0);
    if (rc) return rc;
    st = SolveState();
    st.scale.resize(h.nprob());
    st.rel.assign(h.nprob(), INFINITY);
    st.res.assign(h.nprob(), 0.0);
    h.fstar_max = 0.0;
    for (int p = 0; p < h.nprob(); ++p) {
        st.scale[p] = h.fstar[p] > 0.0 ? h.fstar[p] : 1.0;
        h.fstar_max = std::max(h.fstar_max, h.fstar[p]);
    }
    return MRP_OK;
}

// FP64 composite residual: max |f* - L u| over the leaves of every level
// (level 0 with the exterior ring of the last convolution) into slot 1.
void leaf_residual_launch(Handle& h, cudaStream_t s) {
    cudaMemsetAsync(h.slot(1), 0, sizeof(unsigned long long) * h.nprob(), s);
    for (int k = h.L; k >= 1; --k) inject_level<double>(h, k, s);
    for (int k = h.L; k >= 0; --k) {
        PhaseScope ps(h, s, PH_NORM, h.lv[k].nleaf * n3(h), h.lv[k].nleaf > 0 ? 1 : 0);
        const double hk = level_h(h, k);
        launch_leafres_fused(nullptr, h.lv[k].U, h.lv[k].F, ucoarse<double>(h, k), h.lv[k].leaf_blocks, h.lv[k].nleaf,
                             h.lv[k].view(), view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), h.slot(1),
                             h.nt_leafres[k], s);
    }
}

// Mixed precision, iterative refinement: FP64 outer residual of the composite
// system (leaf rows, and on covered level-0 nodes the mismatch c0 between the
// convolution of the accumulated FP64 source and the injection of level 1),
// FP32 correction cycles from zero, FP64 accumulation.
void outer_residual_launch(Handle& h, cudaStream_t s) {
    Level& l0 = h.lv[0];
    const double inv_h02 = 1.0 / (h.h0 * h.h0);
    coarse_solve<double>(h, s);
    cudaMemsetAsync(h.slot(1), 0, sizeof(unsigned long long) * h.nprob(), s);
    for (int k = h.L; k >= 2; --k) inject_level<double>(h, k, s);
    if (h.L >= 1) {
        PhaseScope ps(h, s, PH_NORM, l0.ncov * n3(h), l0.ncov > 0 ? 1 : 0);
        launch_c0(h.c0, h.off32, l0.U, h.lv[1].U, l0.cov_blocks, l0.ncov, l0.children, h.n, inv_h02, h.slot(1), l0.prob, s);
    }
    for (int k = 1; k <= h.L; ++k) {
        PhaseScope ps(h, s, PH_NORM, h.lv[k].nleaf * n3(h), h.lv[k].nleaf > 0 ? 1 : 0);
        const double hk = level_h(h, k);
        // the residual rows go straight into the FP32 right-hand side of the next correction
        launch_leafres_fused(h.lv[k].F32, h.lv[k].U, h.lv[k].F, ucoarse<double>(h, k), h.lv[k].leaf_blocks, h.lv[k].nleaf,
                             h.lv[k].view(), view_or_empty(h, k - 1), h.n, h.M, 1.0 / (hk * hk), h.slot(1),
                             h.nt_leafres[k], s);
    }
}

// First refinement step, from u = 0: the FP32 cycles solve the problem itself
// (f* on the leaves of every level, level 0 included; no offset on the
// level-1 -> 0 injection), and the FP64 state takes their result (u on levels
// >= 1, the level-0 source on covered nodes).  The correction from u = 0
// solves the problem itself, so no FP64 residual precedes this step.
void first_step_launch(Handle& h, cudaStream_t s) {
    const size_t S = h.n + 2;
    Level& l0 = h.lv[0];
    {
        PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, h.L + 1);
        for (int k = 0; k <= h.L; ++k)
            launch_cast_rhs(h.lv[k].F32, h.lv[k].F, h.lv[k].leaf_blocks, h.lv[k].nleaf, h.n, false, s);
    }
    cudaMemsetAsync(h.off32, 0, sizeof(float) * l0.nb * n3(h), s);
    for (int k = 0; k <= h.L; ++k) cudaMemsetAsync(h.lv[k].U32, 0, sizeof(float) * h.lv[k].nb * S * S * S, s);
    for (int c = 0; c < h.inner_cycles; ++c) vcycle<float>(h, s);
    PhaseScope ps(h, s, PH_OTHER, h.total_nodes, h.L + 1);
    for (int k = 1; k <= h.L; ++k) launch_accumulate_u(h.lv[k].U, h.lv[k].U32, h.lv[k].nb, h.n, s);
    launch_accumulate_f(l0.F, l0.F32, l0.cov_blocks, l0.ncov, h.n, s);
}

void correction_launch(Handle& h, cudaStream_t s) {
    const size_t S = h.n + 2;
    Level& l0 = h.lv[0];
    {
        // leaf rows of levels >= 1: written by the outer residual; level-0 leaves are exact
        PhaseScope ps(h, s, PH_OTHER, l0.nleaf * n3(h), 1);
        launch_cast_rhs(l0.F32, nullptr, l0.leaf_blocks, l0.nleaf, h.n, true, s);
    }
    for (int k = 0; k <= h.L; ++k) cudaMemsetAsync(h.lv[k].U32, 0, sizeof(float) * h.lv[k].nb * S * S * S, s);
    for (int c = 0; c < h.inner_cycles; ++c) vcycle<float>(h, s);
    PhaseScope ps(h, s, PH_OTHER, h.total_nodes, h.L + 1);
    for (int k = 1; k <= h.L; ++k) launch_accumulate_u(h.lv[k].U, h.lv[k].U32, h.lv[k].nb, h.n, s);
    launch_accumulate_f(l0.F, l0.F32, l0.cov_blocks, l0.ncov, h.n, s);
}

// Cauchy stop rule (Sec. 3): per problem, max |u - u_prev| over the leaf
// nodes of every level into slot 2 and max |u| into slot 3; u_prev = u.
void cauchy_launch(Handle& h, cudaStream_t s) {
    cudaMemsetAsync(h.slot(2), 0, sizeof(unsigned long long) * 2 * h.nprob(), s);
    for (int k = 0; k <= h.L; ++k) {
        PhaseScope ps(h, s, PH_NORM, h.lv[k].nleaf * n3(h), h.lv[k].nleaf > 0 ? 1 : 0);
        launch_cauchy(h.lv[k].Uprev, h.lv[k].U, h.lv[k].leaf_blocks, h.lv[k].nleaf, h.n, h.slot(2), h.slot(3),
                      h.lv[k].prob, s);
    }
}

static void solve_step(Handle& h, cudaStream_t s, SolveState& st) {
    const bool cauchy = h.stop_rule == MRP_STOP_CAUCHY;
    if (!h.mixed) {
        vcycle<double>(h, s);
        ++st.cycles;
        if (cauchy) cauchy_launch(h, s);
        else leaf_residual_launch(h, s);
        return;
    }
    // (one level: the FP64 level-0 convolution of the outer residual is the
    // whole answer, so the first pass runs no FP32 cycles and counts no step)
    if (st.started || h.L >= 1) {
        if (st.started) correction_launch(h, s);
        else first_step_launch(h, s);
        st.cycles += h.inner_cycles;
        ++st.ir;
    }
    outer_residual_launch(h, s);
    if (cauchy) cauchy_launch(h, s);
    st.started = true;
}

static int solve_check(Handle& h, cudaStream_t s, SolveState& st) {
    const int np = h.nprob();
    const bool cauchy = h.stop_rule == MRP_STOP_CAUCHY;
    std::vector<double> r(np), d(np), u(np);
    int rc = MRP_OK;
    if (!cauchy || h.mixed) rc = read_max(h, s, r.data(), 1);
    if (!rc && cauchy) rc = read_max(h, s, d.data(), 2);
    if (!rc && cauchy) rc = read_max(h, s, u.data(), 3);
    if (rc) { st.rc = rc; st.done = true; return rc; }
    bool all = true;
    for (int p = 0; p < np; ++p) {
        st.res[p] = (!cauchy || h.mixed) ? r[p] / st.scale[p] : 0.0;
        st.rel[p] = cauchy ? d[p] / (u[p] > 0.0 ? u[p] : 1.0) : st.res[p];
        if (!std::isfinite(st.rel[p]) || !std::isfinite(st.res[p])) {
            st.rc = MRP_ERR_NUMERICAL;
            st.done = true;
            return MRP_OK;
        }
        if (!(st.rel[p] < h.tol)) all = false;
    }
    if (all) st.done = true;
    else if (!h.mixed && st.cycles >= h.max_cycles) st.done = true;
    else if (h.mixed && (st.ir >= h.max_ir || st.cycles >= h.max_cycles)) st.done = true;
    return MRP_OK;
}

void solve_end(Handle& h, double* u, cudaStream_t s) {
    PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, 1);
    launch_gather_leaves(h, u, s);
}

}  // namespace mrp

using namespace mrp;


extern "C" {

const char* mrp_error_string(int status) {
    switch (status) {
        case MRP_OK: return "ok";
        case MRP_ERR_INVALID_ARG: return "invalid argument";
        case MRP_ERR_INVALID_FOREST: return "invalid forest";
        case MRP_ERR_CUDA: return "CUDA runtime error";
        case MRP_ERR_OOM: return "device out of memory";
        case MRP_ERR_NOT_CONVERGED: return "not converged within max_cycles";
        case MRP_ERR_TIMEOUT: return "device wait budget exhausted";
        case MRP_ERR_NUMERICAL: return "NaN or Inf in the residual";
        case MRP_ERR_UNSUPPORTED: return "unsupported option";
        case MRP_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the no-allocation entry point";
        default: return "unknown status";
    }
}

static void destroy_handle(mrp_handle* H) {
    graph_release(H);
    for (auto& g : H->g) release(*g);
    for (cudaStream_t st : H->gs) cudaStreamDestroy(st);
    for (cudaEvent_t e : H->ev) cudaEventDestroy(e);
    delete H;
}

int mrp_create(mrp_handle** out, const mrp_forest* forests, int32_t n_forests, const mrp_options* opt) {
    if (!out) return MRP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!forests || !opt || n_forests < 1) return MRP_ERR_INVALID_ARG;
    if (opt->order != 2 && opt->order != 4 && opt->order != 6) return MRP_ERR_INVALID_ARG;
    if (opt->nu1 < 0 || opt->nu2 < 0 || opt->max_cycles < 1 || !(opt->tol >= 0.0)) return MRP_ERR_INVALID_ARG;
    if (opt->stop_rule != MRP_STOP_RESIDUAL && opt->stop_rule != MRP_STOP_CAUCHY) return MRP_ERR_INVALID_ARG;
    if (opt->precision != MRP_FP64 && opt->precision != MRP_MIXED) return MRP_ERR_INVALID_ARG;
    if (opt->inner_cycles < 0 || opt->max_outer < 0) return MRP_ERR_INVALID_ARG;
    {
        const int ct = opt->launch & ~MRP_LAUNCH_NOSTAGE;
        const bool nostage = (opt->launch & MRP_LAUNCH_NOSTAGE) != 0;
        if (opt->launch != 0 && ct != 128 && ct != 256 && (ct != 512 || nostage)) return MRP_ERR_INVALID_ARG;
    }
    // problems (forest, component) in the caller's layout order, grouped by block size
    std::map<int, std::vector<ProblemDesc>> by_n;
    int64_t off = 0;
    for (int i = 0; i < n_forests; ++i) {
        const mrp_forest& f = forests[i];
        if (f.ncomp < 1 || f.n_leaves < 1 || !f.leaf_level || !f.leaf_ijk) return MRP_ERR_INVALID_ARG;
        if (f.n % 2 != 0 || f.n < 8 || f.n > 24) return MRP_ERR_INVALID_FOREST;
        for (int c = 0; c < f.ncomp; ++c) {
            by_n[f.n].push_back(ProblemDesc{&f, i, c, off});
            off += (int64_t)f.n_leaves * f.n * f.n * f.n;
        }
    }
    mrp_handle* H = new (std::nothrow) mrp_handle();
    if (!H) return MRP_ERR_OOM;
    H->elems = off;
    int rc = MRP_OK;
    for (auto& kv : by_n) {
        H->g.emplace_back(new (std::nothrow) Handle());
        if (!H->g.back()) { rc = MRP_ERR_OOM; break; }
        Handle& h = *H->g.back();
        h.M = opt->order; h.nu1 = opt->nu1; h.nu2 = opt->nu2; h.max_cycles = opt->max_cycles;
        h.tol = opt->tol; h.stop_rule = opt->stop_rule;
        h.mixed = opt->precision == MRP_MIXED;
        h.inner_cycles = opt->inner_cycles > 0 ? opt->inner_cycles : 4;
        h.max_ir = opt->max_outer > 0 ? opt->max_outer : 12;
        h.launch_override = opt->launch;
        tune_defaults(h);
        std::string why;
        rc = build_forest(h, kv.second, why);
        if (rc == MRP_OK && (fused_smem_bytes(h.n, h.M, 8) > (size_t)MAX_DYN_SMEM ||
                             (h.mixed && fused_smem_bytes(h.n, h.M, 4) > (size_t)MAX_DYN_SMEM)))
            rc = MRP_ERR_UNSUPPORTED;
        if (rc == MRP_OK) rc = upload_tables(h);
        if (rc == MRP_OK) rc = fft_plan(h);
        if (rc == MRP_OK) rc = lgf_build(h, 0);
        if (rc == MRP_OK && h.mixed) rc = mixed_setup(h);
        if (rc != MRP_OK) break;
    }
    if (rc == MRP_OK && H->g.size() > 1) {
        for (size_t i = 0; i < H->g.size() && rc == MRP_OK; ++i) {
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = MRP_ERR_CUDA;
            else H->gs.push_back(st);
        }
        for (size_t i = 0; i < 1 + H->g.size() && rc == MRP_OK; ++i) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = MRP_ERR_CUDA;
            else H->ev.push_back(e);
        }
    }
    if (rc == MRP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = MRP_ERR_CUDA;
    if (rc != MRP_OK) {
        cudaGetLastError();
        destroy_handle(H);
        return rc;
    }
    *out = H;
    return MRP_OK;
}

int mrp_destroy(mrp_handle* H) {
    if (!H) return MRP_OK;
    destroy_handle(H);
    return MRP_OK;
}

// Streams of the groups: the caller's stream alone for one group; otherwise
// one stream per group, forked from and joined back into the caller's stream.
static std::vector<cudaStream_t> fork_streams(mrp_handle* H, cudaStream_t s) {
    if (H->g.size() == 1) return {s};
    cudaEventRecord(H->ev[0], s);
    for (cudaStream_t gs : H->gs) cudaStreamWaitEvent(gs, H->ev[0], 0);
    return H->gs;
}

static void join_streams(mrp_handle* H, cudaStream_t s) {
    if (H->g.size() == 1) return;
    for (size_t i = 0; i < H->gs.size(); ++i) {
        cudaEventRecord(H->ev[1 + i], H->gs[i]);
        cudaStreamWaitEvent(s, H->ev[1 + i], 0);
    }
}

int mrp_solve(mrp_handle* H, const double* f, double* u, void* stream, mrp_stats* st) {
    if (!H || !f || !u) return MRP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t G = H->g.size();
    std::vector<int64_t> launches0(G);
    for (size_t i = 0; i < G; ++i) launches0[i] = H->g[i]->launches;
    for (size_t i = 0; i < G; ++i)
        if (autotune(*H->g[i], s)) return MRP_ERR_CUDA;
    const std::vector<cudaStream_t> gs = fork_streams(H, s);
    for (size_t i = 0; i < G; ++i) solve_begin(*H->g[i], f, gs[i]);
    std::vector<SolveState> ss(G);
    int rc = MRP_OK;
    for (size_t i = 0; i < G && rc == MRP_OK; ++i) rc = solve_begin_read(*H->g[i], gs[i], ss[i]);
    if (rc) return rc;
    for (;;) {
        bool any = false;
        for (size_t i = 0; i < G; ++i)
            if (!ss[i].done) { solve_step(*H->g[i], gs[i], ss[i]); any = true; }
        if (!any) break;
        for (size_t i = 0; i < G; ++i)
            if (!ss[i].done && solve_check(*H->g[i], gs[i], ss[i]) == MRP_ERR_CUDA) return MRP_ERR_CUDA;
    }
    for (size_t i = 0; i < G; ++i) solve_end(*H->g[i], u, gs[i]);
    join_streams(H, s);
    if (cudaGetLastError() != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    bool converged = true;
    for (size_t i = 0; i < G; ++i) {
        H->g[i]->have_forward = true;
        if (ss[i].rc && !rc) rc = ss[i].rc;
        if (!(ss[i].worst() < H->g[i]->tol)) converged = false;
    }
    if (st) {
        std::memset(st, 0, sizeof(*st));
        for (size_t i = 0; i < G; ++i) {
            const Handle& h = *H->g[i];
            st->cycles = std::max(st->cycles, ss[i].cycles);
            st->ir_steps = std::max(st->ir_steps, ss[i].ir);
            st->residual = std::max(st->residual, ss[i].worst_res());
            if (h.stop_rule == MRP_STOP_CAUCHY) st->cauchy = std::max(st->cauchy, ss[i].worst());
            st->fstar_max = std::max(st->fstar_max, h.fstar_max);
            st->leaf_nodes += h.leaf_nodes;
            st->total_nodes += h.total_nodes;
            st->launches += h.launches - launches0[i];
        }
    }
    if (rc) return rc;
    return converged ? MRP_OK : MRP_ERR_NOT_CONVERGED;
}

int mrp_solve_adjoint(mrp_handle* H, const double* w, double* fbar, void* stream, mrp_stats* st) {
    if (!H || !w || !fbar) return MRP_ERR_INVALID_ARG;
    int rc = MRP_OK;
    if (st) std::memset(st, 0, sizeof(*st));
    for (auto& g : H->g) {
        Handle& h = *g;
        const int64_t launches0 = h.launches;
        int cycles = 0;
        double rel = INFINITY;
        const int r = solve_adjoint(h, w, fbar, (cudaStream_t)stream, &cycles, &rel);
        if (r == MRP_ERR_CUDA || r == MRP_ERR_OOM) return r;
        if (r && (!rc || rc == MRP_ERR_NOT_CONVERGED)) rc = r;
        if (st) {
            st->cycles = std::max(st->cycles, cycles);
            st->ir_steps = st->cycles;
            st->residual = std::max(st->residual, rel);
            st->leaf_nodes += h.leaf_nodes;
            st->total_nodes += h.total_nodes;
            st->launches += h.launches - launches0;
        }
    }
    return rc;
}

int mrp_adjoint_len(mrp_handle* H, int64_t* len) {
    if (!H || !len) return MRP_ERR_INVALID_ARG;
    *len = H->g[0]->total_nodes;
    return MRP_OK;
}

int mrp_adjoint_op(mrp_handle* H, int32_t op, const double* in, double* out, void* stream) {
    if (!H || !in || !out) return MRP_ERR_INVALID_ARG;
    if (H->g.size() != 1) return MRP_ERR_UNSUPPORTED;
    return adjoint_op(*H->g[0], op, in, out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- step API
int mrp_level_count(mrp_handle* H, int32_t* levels) {
    if (!H || !levels) return MRP_ERR_INVALID_ARG;
    *levels = H->g[0]->L + 1;
    return MRP_OK;
}

int mrp_level_info(mrp_handle* H, int32_t level, int32_t* nb, int32_t* coords, uint8_t* is_leaf) {
    if (!H || !nb || level < 0 || level > H->g[0]->L) return MRP_ERR_INVALID_ARG;
    const Level& lv = H->g[0]->lv[level];
    *nb = lv.nb;
    if (coords) std::memcpy(coords, lv.h_coords.data(), sizeof(int32_t) * 3 * lv.nb);
    if (is_leaf) std::memcpy(is_leaf, lv.h_is_leaf.data(), lv.nb);
    return MRP_OK;
}

int mrp_field_copy(mrp_handle* H, int32_t field, int32_t level, double* buf, int32_t to_handle, void* stream) {
    if (!H || !buf || level < 0 || level > H->g[0]->L) return MRP_ERR_INVALID_ARG;
    Handle& h = *H->g[0];
    Level& lv = h.lv[level];
    const size_t n = h.n;
    double* p = nullptr;
    size_t cnt = 0;
    switch (field) {
        case MRP_FIELD_U: p = lv.U; cnt = lv.nb * (n + 2) * (n + 2) * (n + 2); break;
        case MRP_FIELD_F: p = lv.F; cnt = lv.nb * n * n * n; break;
        case MRP_FIELD_R: p = lv.R; cnt = lv.nb * n * n * n; break;
        case MRP_FIELD_UHAT: p = lv.H; cnt = lv.nb * n * n * n; break;
        case MRP_FIELD_FRAW:
            if (!lv.Fraw) return MRP_ERR_UNSUPPORTED;        // kept for order 6 only
            p = lv.Fraw; cnt = lv.nb * (n + 4) * (n + 4) * (n + 4); break;
        default: return MRP_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = to_handle ? cudaMemcpyAsync(p, buf, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s)
                              : cudaMemcpyAsync(buf, p, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
}

int mrp_step(mrp_handle* H, int32_t step, int32_t level, const double* f_leaf, void* stream) {
    if (!H) return MRP_ERR_INVALID_ARG;
    Handle& h = *H->g[0];
    cudaStream_t s = (cudaStream_t)stream;
    const bool lvl_ok = level >= 0 && level <= h.L;
    switch (step) {
        case MRP_STEP_PREPARE_RHS:
            if (!f_leaf) return MRP_ERR_INVALID_ARG;
            prepare_rhs(h, f_leaf, s);
            break;
        case MRP_STEP_GHOST_U:
            if (!lvl_ok) return MRP_ERR_INVALID_ARG;
            ghost_u<double>(h, level, s);
            break;
        case MRP_STEP_SMOOTH:
            if (!lvl_ok) return MRP_ERR_INVALID_ARG;
            smooth<double>(h, level, s);
            break;
        case MRP_STEP_RESIDUAL:
            if (!lvl_ok) return MRP_ERR_INVALID_ARG;
            residual<double>(h, level, s);
            break;
        case MRP_STEP_RESTRICT:
            if (!lvl_ok || level < 1) return MRP_ERR_INVALID_ARG;
            restrict_level<double>(h, level, s);
            break;
        case MRP_STEP_COARSE_SOLVE:
            coarse_solve<double>(h, s);
            break;
        case MRP_STEP_PROLONG:
            if (!lvl_ok || level < 1) return MRP_ERR_INVALID_ARG;
            prolong<double>(h, level, s);
            break;
        case MRP_STEP_VCYCLE:
            vcycle<double>(h, s);
            break;
        case MRP_STEP_COARSE_SOLVE_F32: {
            if (!h.mixed) return MRP_ERR_UNSUPPORTED;
            Level& l0 = h.lv[0];
            launch_block_copy<float, double>(l0.F32, l0.F, l0.order, l0.nb, h.n, 1.0, s);
            coarse_solve<float>(h, s);
            // the (n+2)^3 boxes, widened
            launch_block_copy<double, float>(l0.U, ucur<float>(h, 0), l0.order, l0.nb, h.n + 2, 1.0, s);
            break;
        }
        default:
            return MRP_ERR_INVALID_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
}

int mrp_lgf_extent(mrp_handle* H, int32_t* nmax) {
    if (!H || !nmax) return MRP_ERR_INVALID_ARG;
    *nmax = H->g[0]->lgf_nmax;
    return MRP_OK;
}

int mrp_lgf_copy(mrp_handle* H, int32_t nmax, double* out_host) {
    if (!H || !out_host || nmax < 0 || nmax > H->g[0]->lgf_nmax) return MRP_ERR_INVALID_ARG;
    const int nn = H->g[0]->lgf_nmax + 1, m = nmax + 1;
    std::vector<double> all((size_t)nn * nn * nn);
    if (cudaMemcpy(all.data(), H->g[0]->lgf, sizeof(double) * all.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MRP_ERR_CUDA;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            for (int c = 0; c < m; ++c) out_host[((size_t)a * m + b) * m + c] = all[((size_t)a * nn + b) * nn + c];
    return MRP_OK;
}

int mrp_profile_enable(mrp_handle* H, int32_t enable) {
    if (!H) return MRP_ERR_INVALID_ARG;
    Handle& h = *H->g[0];
    if (enable && h.ev.empty()) {
        h.ev.resize(4096);
        for (auto& e : h.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return MRP_ERR_CUDA;
    }
    h.prof = enable != 0;
    return MRP_OK;
}

int mrp_profile_read(mrp_handle* H, int32_t n, double* ms, int64_t* launches, int64_t* nodes, int32_t reset) {
    if (!H || n < 0 || n > 16) return MRP_ERR_INVALID_ARG;
    Handle& h = *H->g[0];
    if (!h.pend.empty()) {
        if (cudaDeviceSynchronize() != cudaSuccess) return MRP_ERR_CUDA;
        harvest(h);
    }
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = h.prof_ms[i];
        if (launches) launches[i] = h.prof_cnt[i];
        if (nodes) nodes[i] = h.prof_nodes[i];
    }
    if (reset)
        for (int i = 0; i < 16; ++i) { h.prof_ms[i] = 0; h.prof_cnt[i] = 0; h.prof_nodes[i] = 0; }
    return MRP_OK;
}

int mrp_fft_shape(mrp_handle* H, int32_t* P) {
    if (!H || !P) return MRP_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) P[a] = H->g[0]->pr[0].ax[a].P;
    return MRP_OK;
}

}  // extern "C"
