// Merge of groups that span domains (the paper's distributed step, Sec. 3.3,
// Fig. "Distributed Union-Find": steps 3 and 4).
//
// Every domain (one GPU) runs the local group finder on its own particles
// plus a ghost layer of width l_x, labels each local group with a globally
// unique id, and reports links (id_a, id_b) for groups that touch the domain
// boundary.  After the links of all domains are gathered (all-gather), every
// domain runs this union-find over the gathered list:
//   * group ids are mapped to dense indices with a hash table (Sec. 3.4.1,
//     "Hash table": O(1) look-ups instead of searching the list);
//   * sets are joined by size (Sec. 3.3: union-by-size spreads the roots of
//     spanning groups over the domains instead of skewing them towards the
//     lowest ranks); the weight of an id is the number of particles the
//     caller attributes to it (1 when no weights are given);
//   * every set also keeps its smallest id, which is the label reported, so
//     the result does not depend on the order of the links or on the union
//     order (the library labels groups by their smallest particle index).
// Indirect links (a group joined to another only through groups of third
// domains) are followed because the whole gathered list is processed.
//
// Host code only: it needs no GPU and runs where the caller gathers.
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

#include "fof.h"

namespace {

// Open-addressing hash table from a 64-bit id to a dense index.
class IdTable {
public:
    explicit IdTable(size_t expect)
    {
        size_t cap = 16;
        while (cap < 2 * expect + 16) cap <<= 1;
        keys_.assign(cap, kEmpty);
        vals_.assign(cap, -1);
        mask_ = cap - 1;
    }

    // index of id, inserting it (with the next dense index) if absent
    int64_t insert(int64_t id, int64_t next, bool& fresh)
    {
        size_t h = slot(id);
        for (;;) {
            if (keys_[h] == kEmpty) {
                keys_[h] = id;
                vals_[h] = next;
                fresh = true;
                return next;
            }
            if (keys_[h] == id) {
                fresh = false;
                return vals_[h];
            }
            h = (h + 1) & mask_;
        }
    }

    int64_t find(int64_t id) const
    {
        size_t h = slot(id);
        for (;;) {
            if (keys_[h] == kEmpty)
                return -1;
            if (keys_[h] == id)
                return vals_[h];
            h = (h + 1) & mask_;
        }
    }

private:
    static constexpr int64_t kEmpty = INT64_MIN;
    size_t slot(int64_t id) const
    {
        uint64_t x = (uint64_t)id;               // splitmix64 finaliser
        x ^= x >> 30;
        x *= 0xbf58476d1ce4e5b9ULL;
        x ^= x >> 27;
        x *= 0x94d049bb133111ebULL;
        x ^= x >> 31;
        return (size_t)x & mask_;
    }
    std::vector<int64_t> keys_, vals_;
    size_t mask_ = 0;
};

struct Sets {
    std::vector<int64_t> parent, weight, minid;

    int64_t add(int64_t id, int64_t w)
    {
        parent.push_back((int64_t)parent.size());
        weight.push_back(w);
        minid.push_back(id);
        return (int64_t)parent.size() - 1;
    }

    int64_t find(int64_t x)
    {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];        // path halving
            x = parent[x];
        }
        return x;
    }

    void unite(int64_t a, int64_t b)
    {
        a = find(a);
        b = find(b);
        if (a == b)
            return;
        if (weight[a] < weight[b] || (weight[a] == weight[b] && minid[a] > minid[b])) {
            int64_t t = a;
            a = b;
            b = t;
        }
        parent[b] = a;                            // the lighter set joins the heavier
        weight[a] += weight[b];
        if (minid[b] < minid[a])
            minid[a] = minid[b];
    }
};

}  // namespace

extern "C" int fof_merge_links(int64_t npairs, const int64_t* a, const int64_t* b, int64_t nweights,
                               const int64_t* weight_ids, const int64_t* weights, int64_t nq,
                               const int64_t* query, int64_t* label_out, int64_t* weight_out)
{
    if (npairs < 0 || nweights < 0 || nq < 0 || (npairs > 0 && (!a || !b)) ||
        (nweights > 0 && (!weight_ids || !weights)) || (nq > 0 && (!query || !label_out)))
        return FOF_ERR_ARG;
    try {
        IdTable table((size_t)(2 * npairs + nweights));
        Sets sets;
        sets.parent.reserve((size_t)(2 * npairs + nweights));
        sets.weight.reserve((size_t)(2 * npairs + nweights));
        sets.minid.reserve((size_t)(2 * npairs + nweights));
        auto index = [&](int64_t id, int64_t w) {
            bool fresh = false;
            int64_t k = table.insert(id, (int64_t)sets.parent.size(), fresh);
            if (fresh)
                sets.add(id, w);
            return k;
        };
        // weights first, so that every weighted id enters with its weight
        for (int64_t k = 0; k < nweights; ++k) {
            bool fresh = false;
            int64_t i = table.insert(weight_ids[k], (int64_t)sets.parent.size(), fresh);
            if (fresh)
                sets.add(weight_ids[k], weights[k]);
            else
                sets.weight[sets.find(i)] += weights[k];
        }
        for (int64_t k = 0; k < npairs; ++k) {
            const int64_t ia = index(a[k], 1);
            const int64_t ib = index(b[k], 1);
            sets.unite(ia, ib);
        }
        for (int64_t k = 0; k < nq; ++k) {
            const int64_t i = table.find(query[k]);
            if (i < 0) {
                label_out[k] = query[k];
                if (weight_out) weight_out[k] = 0;
            } else {
                const int64_t r = sets.find(i);
                label_out[k] = sets.minid[r];
                if (weight_out) weight_out[k] = sets.weight[r];
            }
        }
    } catch (const std::bad_alloc&) {
        return FOF_ERR_OOM;
    }
    return FOF_OK;
}
