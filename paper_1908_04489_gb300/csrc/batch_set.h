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
    LaunchCfg cfg;                // launch shapes (results do not depend on them)
};

// Descriptor of a fast-path instance from its host-side state.
InstDev describe_inst(const ucp_inst* in);

// Rebuild descriptors and block maps for `members` and upload them on `s`.
ucp_status batchset_build(BatchSet& bs, const std::vector<ucp_inst*>& members,
                          cudaStream_t s);

// Re-upload the descriptors of the same members (pointers, cur, sweeps).
ucp_status batchset_refresh(BatchSet& bs, const std::vector<ucp_inst*>& members,
                            cudaStream_t s);

// Batched set-up of members created without their own (inst_init with
// own_setup = false): weights, coarse list, init, counters, the fast path's
// constants and filter slices (five launches for all members), then the first
// u1 update, tables and J as the rest of one batched sweep (bs built for the
// same members), and the descriptors as the host sees them.
struct SetupSet {
    Arena* arena = nullptr;
    SetupDev* descs = nullptr;
    size_t descs_cap = 0;
    BlockRef* maps = nullptr;
    size_t maps_cap = 0;
    std::vector<SetupDev> desc;
    std::vector<BlockRef> host_maps;
};
ucp_status batchset_setup(SetupSet& ss, BatchSet& bs, const std::vector<ucp_inst*>& members,
                          cudaStream_t s);

}  // namespace ucp
