// Pair kernels (descriptor forward, force backward) for K = 32 radial
// channels: the instances of pair_kernels.cuh for every supported species count.
#include "pair_kernels.cuh"

namespace tmd {

TMD_PAIR_LAUNCHER(launch_pair_k32) {
    switch (dm.S) {
    case 1: return launch_pair_kernels<32, 1>(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 2: return launch_pair_kernels<32, 2>(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 3: return launch_pair_kernels<32, 3>(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 4: return launch_pair_kernels<32, 4>(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 5: return launch_pair_kernels<32, 5>(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    default: break;
    }
    set_error("no kernel for K=%d S=%d", dm.K, dm.S);
    return TMD_ERR_UNIMPLEMENTED;
}

}  // namespace tmd
