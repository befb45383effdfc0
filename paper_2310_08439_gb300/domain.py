"""Spatial domain decomposition of one periodic system (the paper's MPI
scheme for its strong- and weak-scaling runs, Sec. "Evaluation").

The box is cut into R slabs along x, one per rank.  A rank owns the atoms of
its slab and evaluates their energy terms; the atoms of the neighbouring
slabs within the halo width h (>= the table radius rc + skin) of its faces
come in as ghosts (forward exchange of positions), placed at the image
positions they have next to the slab.  The TensorMD energy of an atom depends
on all its neighbours, so a pair (i, j) with i owned and j a ghost puts a
force on j that belongs to j's owner: those ghost forces go back (reverse
exchange) and are added there.  Energy and virial are FP64 sums over owned
centres, all-reduced over the ranks.  With the halo of one table radius and
the reverse exchange, every pair is evaluated exactly once, by the owner of
its centre atom, and the totals are those of the whole box.

The per-rank force call is an ``engine(pos, types, n_owned, box, pbc)``
returning (energy of the owned centres, forces [n, 3] of owned atoms and
ghosts, virial [3, 3]).  ``gpu_engine`` builds it on the library's
tmd_compute_owned; the protocol itself is plain host code (NumPy plus a
``comm`` that moves arrays between ranks: torch.distributed in
``TorchComm``, or every rank in one process in ``evaluate_serial``).
"""
from __future__ import annotations

import numpy as np

# positions of a slab's atoms in its local frame start this far inside the
# local box (rounding of x - lo never leaves it)
_EDGE = 1e-6


class Slabs:
    """R slabs along x of an orthorhombic box; the halo h must not exceed a
    slab's width (ghosts then come from the two neighbouring slabs only)."""

    def __init__(self, box, pbc, n_ranks, halo):
        self.box = np.asarray(box, dtype=np.float64)
        self.pbc = np.asarray(pbc, dtype=np.int32)
        self.R = int(n_ranks)
        self.h = float(halo)
        self.w = self.box[0] / self.R
        if self.R < 1 or self.h <= 0.0:
            raise ValueError("need >= 1 rank and a positive halo")
        if self.w < self.h:
            raise ValueError(f"slab width {self.w:.3f} A is below the halo {self.h:.3f} A: use fewer ranks")
        if self.R > 1 and not self.pbc[0]:
            raise ValueError("slabs along a non-periodic axis are not supported")

    def bounds(self, r):
        return r * self.w, (r + 1) * self.w

    def owner(self, x):
        """Rank owning positions x (wrapped into the box on x)."""
        r = np.floor(np.mod(x, self.box[0]) / self.w).astype(np.int64)
        return np.clip(r, 0, self.R - 1)

    def local_box(self):
        b = self.box.copy()
        b[0] = self.w + 2.0 * self.h + 2.0 * _EDGE
        return b

    def local_pbc(self):
        p = self.pbc.copy()
        p[0] = 0
        return p


class Domain:
    """One rank's atoms: global ids, positions (wrapped on x into its slab),
    velocities, species, masses."""

    def __init__(self, slabs, rank, gid, pos, vel, types, mass):
        self.s, self.r = slabs, int(rank)
        self.lo, self.hi = slabs.bounds(self.r)
        self.gid = np.asarray(gid, dtype=np.int64)
        self.pos = np.array(pos, dtype=np.float64).reshape(-1, 3)
        self.vel = np.array(vel, dtype=np.float64).reshape(-1, 3)
        self.types = np.asarray(types, dtype=np.int32)
        self.mass = np.asarray(mass, dtype=np.float64)

    @property
    def n(self):
        return self.gid.size


def split(slabs, pos, vel, types, mass):
    """The R domains of a whole system (positions wrapped on x)."""
    pos = np.array(pos, dtype=np.float64)
    pos[:, 0] = np.mod(pos[:, 0], slabs.box[0])
    own = slabs.owner(pos[:, 0])
    out = []
    for r in range(slabs.R):
        k = np.nonzero(own == r)[0]
        out.append(Domain(slabs, r, k, pos[k], np.asarray(vel)[k], np.asarray(types)[k], np.asarray(mass)[k]))
    return out


def ghost_sends(d):
    """What rank d.r sends: (to_left, to_right), each (indices into its atoms,
    positions as the receiver places them).  Atoms within h of the low face
    go left, within h of the high face go right; across the periodic end of
    the box the positions move by one box length."""
    s = d.s
    L = s.box[0]
    x = d.pos[:, 0]
    il = np.nonzero(x < d.lo + s.h)[0]
    ir = np.nonzero(x >= d.hi - s.h)[0]
    pl = d.pos[il].copy()
    pr = d.pos[ir].copy()
    if d.r == 0:
        pl[:, 0] += L          # the left neighbour of rank 0 sits below x = L
    if d.r == s.R - 1:
        pr[:, 0] -= L          # the right neighbour of the last rank sits above x = 0
    return (il, pl), (ir, pr)


def assemble(d, from_left, from_right):
    """Local arrays of rank d.r: owned atoms first, then the ghosts from the
    left and from the right (positions, species); x shifted into the local
    box [0, w + 2 h)."""
    (tl, pl), (tr, pr) = from_left, from_right
    pos = np.concatenate([d.pos, pl, pr]).copy()
    types = np.concatenate([d.types, tl, tr]).astype(np.int32)
    pos[:, 0] += d.s.h + _EDGE - d.lo
    return pos, types


def ghost_forces(d, F, n_left):
    """Split the forces of the local atoms: owned, back to the left, back to
    the right."""
    n = d.n
    return F[:n], F[n:n + n_left], F[n + n_left:]


def evaluate_serial(slabs, domains, engine):
    """Every rank of the protocol in one process (the exchanges are array
    copies): returns (E, per-domain owned forces, W)."""
    R = slabs.R
    sends = [ghost_sends(d) for d in domains]
    E, W, forces = 0.0, np.zeros((3, 3)), [np.zeros((d.n, 3)) for d in domains]
    back = []
    for r, d in enumerate(domains):
        left, right = domains[(r - 1) % R], domains[(r + 1) % R]
        (il_r, pl_r) = sends[(r - 1) % R][1]     # the left neighbour's high-face atoms
        (ir_l, pr_l) = sends[(r + 1) % R][0]     # the right neighbour's low-face atoms
        pos, types = assemble(d, (left.types[il_r], pl_r), (right.types[ir_l], pr_l))
        e, F, w = engine(pos, types, d.n, slabs.local_box(), slabs.local_pbc())
        E += e
        W += w
        own, fl, fr = ghost_forces(d, F, il_r.size)
        forces[r] += own
        back.append((fl, fr))
    for r in range(R):
        # ghosts of rank r from its left came from that rank's high face, and so on
        fl, fr = back[r]
        forces[(r - 1) % R][sends[(r - 1) % R][1][0]] += fl
        forces[(r + 1) % R][sends[(r + 1) % R][0][0]] += fr
    return E, forces, W


class TorchComm:
    """Exchanges between neighbouring ranks over torch.distributed (gloo for
    host arrays; with NCCL the arrays travel as device tensors)."""

    def __init__(self, dist, device="cpu"):
        self.dist, self.device = dist, device
        self.rank, self.size = dist.get_rank(), dist.get_world_size()

    def _t(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a)).to(self.device)

    def sendrecv(self, to_left, to_right):
        """Send to_left to rank - 1 and to_right to rank + 1 (periodic), receive
        (from_left, from_right); each payload is a list of NumPy arrays whose
        dtypes and trailing shapes both sides agree on."""
        import torch
        R = self.size
        if R == 1:
            return to_right, to_left          # the rank is its own neighbour on both sides
        left, right = (self.rank - 1) % R, (self.rank + 1) % R
        d = self.dist
        # lengths first
        ln = [self._t(np.array([a.shape[0] for a in to_left], dtype=np.int64)),
              self._t(np.array([a.shape[0] for a in to_right], dtype=np.int64))]
        got = [torch.zeros(len(to_right), dtype=torch.int64, device=self.device),
               torch.zeros(len(to_left), dtype=torch.int64, device=self.device)]
        self._pairwise(ln, got, left, right, tag=0)
        n_from_left, n_from_right = got[0].cpu().numpy(), got[1].cpu().numpy()
        from_left, from_right = [], []
        for q, (al, ar) in enumerate(zip(to_left, to_right)):
            rl = torch.zeros((int(n_from_left[q]),) + al.shape[1:], dtype=self._t(al).dtype, device=self.device)
            rr = torch.zeros((int(n_from_right[q]),) + ar.shape[1:], dtype=self._t(ar).dtype, device=self.device)
            self._pairwise([self._t(al), self._t(ar)], [rl, rr], left, right, tag=1 + q)
            from_left.append(rl.cpu().numpy())
            from_right.append(rr.cpu().numpy())
        return from_left, from_right

    def _pairwise(self, send, recv, left, right, tag):
        """send[0] -> left, send[1] -> right; recv[0] <- left, recv[1] <- right.
        Every rank receives from its left first and sends to its right first,
        so that with two ranks (each the other's left and right) the messages
        pair up in order even where tags are ignored; empty arrays (whose
        length both sides know) are not sent."""
        d = self.dist
        ops = []
        if recv[0].numel():
            ops.append(d.irecv(recv[0], src=left, tag=2 * tag))
        if recv[1].numel():
            ops.append(d.irecv(recv[1], src=right, tag=2 * tag + 1))
        if send[1].numel():
            ops.append(d.isend(send[1], dst=right, tag=2 * tag))
        if send[0].numel():
            ops.append(d.isend(send[0], dst=left, tag=2 * tag + 1))
        for op in ops:
            op.wait()

    def allreduce_sum(self, a):
        t = self._t(np.asarray(a, dtype=np.float64))
        self.dist.all_reduce(t)
        return t.cpu().numpy()


class LocalComm:
    """The exchanges of a single rank (its own neighbour on both sides)."""

    def sendrecv(self, to_left, to_right):
        return to_right, to_left

    def allreduce_sum(self, a):
        return np.asarray(a, dtype=np.float64)


def evaluate(comm, d, engine):
    """This rank's share of one decomposed evaluation: the owned atoms'
    forces [n_owned, 3] and the all-reduced (E, W [3, 3])."""
    (il, pl), (ir, pr) = ghost_sends(d)
    fl, fr = comm.sendrecv([d.types[il], pl], [d.types[ir], pr])
    pos, types = assemble(d, (fl[0], fl[1]), (fr[0], fr[1]))
    e, F, w = engine(pos, types, d.n, d.s.local_box(), d.s.local_pbc())
    own, back_l, back_r = ghost_forces(d, F, fl[0].shape[0])
    # reverse: the forces on ghosts from the left go back left, and so on
    ret_l, ret_r = comm.sendrecv([back_l], [back_r])
    forces = own.copy()
    np.add.at(forces, il, ret_l[0])      # from the left rank: forces on what this rank sent left
    np.add.at(forces, ir, ret_r[0])
    tot = comm.allreduce_sum(np.concatenate([[e], np.asarray(w, dtype=np.float64).ravel()]))
    return forces, float(tot[0]), tot[1:].reshape(3, 3)


def migrate(comm, d):
    """After the drift: atoms that left the slab go to the neighbour whose
    slab they entered (the halo keeps moves to one neighbour per step)."""
    s = d.s
    L = s.box[0]
    d.pos[:, 0] = np.mod(d.pos[:, 0], L)
    own = s.owner(d.pos[:, 0])
    go_l = own == (d.r - 1) % s.R
    go_r = (own == (d.r + 1) % s.R) & ~go_l
    stay = ~(go_l | go_r)
    if s.R > 1 and np.any(own[~stay & ~go_l & ~go_r] != d.r):
        raise RuntimeError("an atom moved further than one slab in one step")
    pack = lambda m: [d.gid[m], d.pos[m], d.vel[m], d.types[m], d.mass[m]]
    fl, fr = comm.sendrecv(pack(go_l), pack(go_r)) if s.R > 1 else ([a[:0] for a in pack(go_l)],
                                                                      [a[:0] for a in pack(go_r)])
    keep = pack(stay)
    parts = [np.concatenate([keep[q], fl[q], fr[q]]) for q in range(5)]
    order = np.argsort(parts[0], kind="stable")   # owned atoms in global-id order
    d.gid, d.pos, d.vel, d.types, d.mass = (p[order] for p in parts)
    d.pos = d.pos.reshape(-1, 3)
    d.vel = d.vel.reshape(-1, 3)


def gpu_engine(tmd, model, torch, r_list, stream=None):
    """Per-rank force call on the library: table over owned atoms and ghosts,
    tmd_compute_owned.  Returns engine(pos, types, n_owned, box, pbc)."""
    nl = tmd.NeighborList()

    def engine(pos, types, n_owned, box, pbc):
        p = torch.as_tensor(pos, dtype=torch.float64, device="cuda")
        t = torch.as_tensor(types, dtype=torch.int32, device="cuda")
        nl.build(p, t, box, pbc, r_list)
        n = p.shape[0]
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        f = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        w = torch.zeros(9, dtype=torch.float64, device="cuda")
        tmd.compute_owned(model, nl, p, t, n_owned, box, energy=e, forces=f, virial=w, stream=stream)
        torch.cuda.synchronize()
        return float(e.item()), f.double().cpu().numpy(), w.cpu().numpy().reshape(3, 3)

    return engine
