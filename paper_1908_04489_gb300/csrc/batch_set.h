// batch_set.h -- descriptors and block maps of a set of fast-path instances
// swept together (used by ucp_batch and by the serving loop).
#pragma once

#include <vector>

#include "ucp_fast.cuh"
#include "ucp_runtime.h"

namespace ucp {

struct BatchSet {
    Arena* arena = nullptr;       // owner of the device buffers below
    InstDev* insts = nullptr;     // [capacity]
    size_t insts_cap = 0;
    BlockRef* maps = nullptr;     // all block maps, back to back
    size_t maps_cap = 0;
    std::vector<InstDev> desc;
    std::vector<BlockRef> host_maps;
    BatchLaunch bl{};
};

// Descriptor of a fast-path instance from its host-side state.
InstDev describe_inst(const ucp_inst* in);

// Rebuild descriptors and block maps for `members` and upload them on `s`.
ucp_status batchset_build(BatchSet& bs, const std::vector<ucp_inst*>& members,
                          cudaStream_t s);

// Re-upload the descriptors of the same members (pointers, cur, sweeps).
ucp_status batchset_refresh(BatchSet& bs, const std::vector<ucp_inst*>& members,
                            cudaStream_t s);

// The set-up step of members created without it (inst_init with
// first_step = false): the first u1 update, tables and J of every member in
// one batched launch, then the descriptors as the host sees them.
ucp_status batchset_first_step(BatchSet& bs, const std::vector<ucp_inst*>& members,
                               cudaStream_t s);

}  // namespace ucp
