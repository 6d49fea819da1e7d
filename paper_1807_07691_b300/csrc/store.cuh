// The device-resident SM store (Sec. 5): per predicate, the matrix M_h laid
// out twice -- rows by subject (side 0, CSR) and rows by object (side 1,
// CSC) -- with the non-zero-row auxiliary arrays of Sec. 6.3 (Row, Rpos;
// Num is the difference of consecutive Rpos) and, for predicates dense
// enough to pay for it, a direct row pointer indexed by entity id.
#pragma once

#include <vector>

#include "common.cuh"
#include "join.cuh"

struct gsmat_store {
    int64_t n_input = 0;
    int64_t n_unique = 0;
    int32_t n_pred = 0;
    int32_t max_entity = -1;
    int32_t max_pred = -1;
    int32_t n_dense[2] = {0, 0};
    int device = 0;

    std::vector<int32_t> pred_ids;          // ascending; index = predicate slot
    std::vector<gs::PredSide> side[2];      // per predicate slot
    std::vector<int32_t> hash_keys;         // open addressing: predicate id or -1
    std::vector<int32_t> hash_vals;         // slot
    uint32_t hash_mask = 0;

    gs::DevBuf key[2], val[2], rowid[2], rowoff[2], dense[2];
    gs::DevBuf pred_side_dev;  // PredSide[2][n_pred] (device copy)
    gs::DevBuf hash_dev;       // int32 keys[cap], vals[cap] (device copy of the hash index)
    gs::StoreView view{};
    gs::TileConfig tiles;  // tile shapes of the plain path's joins on this store

    int64_t device_bytes() const {
        int64_t b = 0;
        for (int s = 0; s < 2; ++s) {
            b += key[s].bytes + val[s].bytes + rowid[s].bytes + rowoff[s].bytes + dense[s].bytes;
        }
        return b + pred_side_dev.bytes + hash_dev.bytes;
    }

    // Predicate hash index lookup on the host: slot or -1.
    int32_t slot_of(int32_t pred_id) const;
};

namespace gs {

uint32_t pred_hash(int32_t p);

int store_build(const int32_t *triples, int64_t n, int on_device, cudaStream_t st, gsmat_store **out);

}  // namespace gs
