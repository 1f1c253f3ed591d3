// tsqs_k16.cu -- kernel instantiations for 16-byte keys.
#include "tsqs_kernels.cuh"
#include "tsqs_task.cuh"

namespace tsqs {

namespace {
constexpr int kLeafBlock = 256, kLeafMaxE = 16, kPivotBlock = 256;
constexpr int kTaskBlock = 256, kTaskItems = 4;   // task schedule: 16 KB tiles

template <int KIND, int BLOCK, int ITEMS, int NBUF>
PartVariant part_variant() {
    PartVariant v;
    v.k_partition = (const void *)k_partition<KIND, BLOCK, ITEMS, NBUF>;
    v.tile = BLOCK * ITEMS;
    v.threads = BLOCK + 32;
    v.smem = (int)PartLayout<KIND, BLOCK, ITEMS, NBUF>::bytes;
    v.nbuf = NBUF;
    return v;
}

template <int KIND>
KindOps make_ops() {
    KindOps o{};
    o.kind = KIND;
    o.elem_size = 16;
    o.leaf_block = kLeafBlock;
    o.pivot_block = kPivotBlock;
    o.leaf_smem = (int)LeafLayout<KIND>::bytes;
    o.leaf_max = kMaxSmall;
    o.part[0] = part_variant<KIND, 192, 6, 3>();
    o.part[1] = part_variant<KIND, 192, 8, 3>();
    o.part[2] = part_variant<KIND, 256, 6, 3>();
    o.part[3] = part_variant<KIND, 256, 4, 3>();
    o.k_init = (const void *)k_init<KIND>;
    o.k_orient = (const void *)k_orient<KIND>;
    o.k_orient_if = (const void *)k_orient_if<KIND>;
    o.k_check = (const void *)k_check<KIND>;
    o.k_presort = (const void *)k_presort<KIND>;
    o.k_deep_prep = (const void *)k_deep_prep<KIND>;
    o.k_deep_tiles = (const void *)k_deep_tiles<KIND>;
    o.k_deep_stage = (const void *)k_deep_stage<KIND>;
    o.k_deep_finish = (const void *)k_deep_finish<KIND>;
    o.k_deep_all = (const void *)k_deep_all<KIND>;
    o.deep_smem = (int)((kDeepTile + kDeepTile / kPadGroup<typename Key<KIND>::C>) * sizeof(typename Key<KIND>::C));
    o.k_leaf = (const void *)k_leaf<KIND, kLeafBlock, kLeafMaxE, 2>;
    o.k_leaf_small = o.k_leaf;
    o.leaf_small_block = o.leaf_block;
    o.leaf_small_smem = o.leaf_smem;
    o.k_pivot = (const void *)k_pivot<KIND>;
    o.k_finish = (const void *)k_level_end<KIND>;
    o.k_dbg_setup_partition = (const void *)k_dbg_setup_partition<KIND>;
    o.k_dbg_counts = (const void *)k_dbg_counts;
    o.k_dbg_pivot = (const void *)k_dbg_pivot<KIND>;
    o.k_task_init = (const void *)k_task_init<KIND>;
    o.k_task = (const void *)k_task<KIND, kTaskBlock, kTaskItems>;
    o.task_block = kTaskBlock;
    o.task_tile = kTaskBlock * kTaskItems;
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
