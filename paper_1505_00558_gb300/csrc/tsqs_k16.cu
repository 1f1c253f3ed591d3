// tsqs_k16.cu -- kernel instantiations for 16-byte keys.
#include "tsqs_kernels.cuh"

namespace tsqs {

namespace {
constexpr int kPartBlock = 256, kItems = 4, kTile = kPartBlock * kItems;
constexpr int kLeafBlock = 256, kPivotBlock = 256, kNBuf = 3;

template <int KIND>
KindOps make_ops() {
    KindOps o{};
    o.kind = KIND;
    o.elem_size = 16;
    o.tile = kTile;
    o.part_block = kPartBlock;
    o.part_threads = kPartBlock + 32;
    o.part_smem = (int)PartLayout<KIND, kPartBlock, kItems, kNBuf>::bytes;
    o.leaf_block = kLeafBlock;
    o.pivot_block = kPivotBlock;
    o.leaf_smem = (kMaxSmall + kMaxSmall / 32) * (int)sizeof(typename Key<KIND>::C);
    o.k_init = (const void *)k_init<KIND, kTile>;
    o.k_leaf = (const void *)k_leaf<KIND, kLeafBlock, 1>;
    o.k_pivot = (const void *)k_pivot<KIND, kTile>;
    o.k_partition = (const void *)k_partition<KIND, kPartBlock, kItems, kNBuf>;
    o.k_finish = (const void *)k_level_end<KIND, kTile>;
    o.k_dbg_setup_partition = (const void *)k_dbg_setup_partition<KIND, kTile>;
    o.k_dbg_counts = (const void *)k_dbg_counts;
    o.k_dbg_pivot = (const void *)k_dbg_pivot<KIND>;
    return o;
}
}  // namespace

const KindOps *ops_k16(int kind) {
    static const KindOps o_TSQS_U64_U64_REC = make_ops<TSQS_U64_U64_REC>();
    switch (kind) {
    case TSQS_U64_U64_REC: return &o_TSQS_U64_U64_REC;
    default: return nullptr;
    }
}

}  // namespace tsqs
