// tsqs_k8.cu -- kernel instantiations for 8-byte keys.
#include "tsqs_kernels.cuh"

namespace tsqs {

namespace {
constexpr int kPartBlock = 256, kItems = 8, kTile = kPartBlock * kItems;
constexpr int kLeafBlock = 256, kPivotBlock = 256, kNBuf = 3;

template <int KIND>
KindOps make_ops() {
    KindOps o{};
    o.kind = KIND;
    o.elem_size = 8;
    o.tile = kTile;
    o.part_block = kPartBlock;
    o.part_threads = kPartBlock + 32;
    o.part_smem = (int)PartLayout<KIND, kPartBlock, kItems, kNBuf>::bytes;
    o.leaf_block = kLeafBlock;
    o.pivot_block = kPivotBlock;
    o.leaf_smem = (kMaxSmall + kMaxSmall / 32) * (int)sizeof(typename Key<KIND>::C);
    o.k_init = (const void *)k_init<KIND, kTile>;
    o.k_leaf = (const void *)k_leaf<KIND, kLeafBlock, 2>;
    o.k_pivot = (const void *)k_pivot<KIND, kTile>;
    o.k_partition = (const void *)k_partition<KIND, kPartBlock, kItems, kNBuf>;
    o.k_finish = (const void *)k_level_end<KIND, kTile>;
    o.k_dbg_setup_partition = (const void *)k_dbg_setup_partition<KIND, kTile>;
    o.k_dbg_counts = (const void *)k_dbg_counts;
    o.k_dbg_pivot = (const void *)k_dbg_pivot<KIND>;
    return o;
}
}  // namespace

const KindOps *ops_k8(int kind) {
    static const KindOps o_TSQS_I64 = make_ops<TSQS_I64>();
    static const KindOps o_TSQS_U64 = make_ops<TSQS_U64>();
    static const KindOps o_TSQS_F64 = make_ops<TSQS_F64>();
    switch (kind) {
    case TSQS_I64: return &o_TSQS_I64;
    case TSQS_U64: return &o_TSQS_U64;
    case TSQS_F64: return &o_TSQS_F64;
    default: return nullptr;
    }
}

}  // namespace tsqs
