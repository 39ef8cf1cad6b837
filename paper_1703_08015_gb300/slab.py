"""Domain split of one geometry across ranks: slabs of tile layers with a
one-tile ghost layer (not in the paper, which names multi-GPU runs as future
work in Sec. 5).

The slowest tile axis (z in 3D, y in 2D) is cut into `world` slabs of whole
tile layers.  Each rank tiles and steps its own box: its slab plus one ghost
tile layer on each side that has a neighbour rank (wrapping around a
periodic axis).  The box is non-periodic along the split axis; its outermost
ghost nodes see a wall there and take wrong values, which the exchange
overwrites.  After every step each rank sends its first and last interior
layers to the neighbours, where they replace the ghost layers, before the
next step reads them.  A node of the slab therefore gathers exactly what it
gathers in the undivided domain, and the split run reproduces the
single-domain run bit for bit.

The tiles of one layer are consecutive in the tile numbering (row-major,
split axis slowest), so a layer is one contiguous byte range of a PDF copy
(``lbm_layer_range``), and the same global layer has the same bytes on the
sending and the receiving rank: the exchange is a plain copy of that range,
NCCL send/recv into the receiver's own memory.  Statistics sum the interior
layers (``lbm_moments_layers``) and are all-reduced over the ranks.

``plan`` and ``box_mask`` are pure host logic; ``SlabSolver`` is the GPU
path.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbm


def split_axis_len(mask: np.ndarray, lattice: int) -> int:
    """Nodes along the split axis (z in 3D, y in 2D) of a [z][y][x] mask."""
    m = np.asarray(mask)
    if m.ndim == 2:
        m = m[None]
    return m.shape[0] if lattice == lbm.LBM_D3Q19 else m.shape[1]


def plan(n_layers: int, world: int, periodic: bool):
    """Per rank, the split of `n_layers` tile layers into `world` slabs.

    Returns a list of dicts, one per rank:
      lo, hi      the rank's interior layers [lo, hi) (global indices);
      lower_rank, upper_rank   neighbour ranks (None at a non-periodic end);
      ghost_lo, ghost_hi       global layer held as a ghost below / above
                               (None where there is no neighbour);
      box         global layers of the rank's box, in box order;
      interior    the interior's local layers [b, e) within the box;
      send        [(peer, local layer, global layer)]: interior layers to send
                  each step;
      recv        [(peer, local layer, global layer)]: ghost layers to receive.
    Both lists are sorted by (peer, global layer), so two ranks that exchange
    two layers with each other (two ranks around a periodic axis) post them
    in the same order, as NCCL's in-order matching of a peer pair needs.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    if world > n_layers:
        raise ValueError(f"{world} ranks for {n_layers} tile layers: every rank needs one layer")
    base, extra = divmod(n_layers, world)
    bounds = [0]
    for r in range(world):
        bounds.append(bounds[-1] + base + (1 if r < extra else 0))
    out = []
    for r in range(world):
        lo, hi = bounds[r], bounds[r + 1]
        has_lower = world > 1 and (r > 0 or periodic)
        has_upper = world > 1 and (r < world - 1 or periodic)
        lower = (r - 1) % world if has_lower else None
        upper = (r + 1) % world if has_upper else None
        g_lo = (lo - 1) % n_layers if has_lower else None
        g_hi = hi % n_layers if has_upper else None
        box = ([g_lo] if has_lower else []) + list(range(lo, hi)) + ([g_hi] if has_upper else [])
        b = 1 if has_lower else 0
        e = b + (hi - lo)
        send, recv = [], []
        if has_lower:
            send.append((lower, b, lo))          # my first interior layer -> their upper ghost
            recv.append((lower, 0, g_lo))        # their last interior layer -> my lower ghost
        if has_upper:
            send.append((upper, e - 1, hi - 1))  # my last interior layer -> their lower ghost
            recv.append((upper, e, g_hi))        # their first interior layer -> my upper ghost
        send.sort(key=lambda t: (t[0], t[2]))
        recv.sort(key=lambda t: (t[0], t[2]))
        out.append({"lo": lo, "hi": hi, "lower_rank": lower, "upper_rank": upper, "ghost_lo": g_lo,
                    "ghost_hi": g_hi, "box": box, "interior": (b, e), "send": send, "recv": recv})
    return out


def box_mask(mask: np.ndarray, lattice: int, tile_a: int, part: dict) -> np.ndarray:
    """The rank's box: the global mask's node rows of `part['box']` layers,
    stacked in box order ([z][y][x]; 2D masks keep nz = 1)."""
    m = np.asarray(mask, np.uint8)
    two_d = m.ndim == 2 or lattice == lbm.LBM_D2Q9
    if m.ndim == 2:
        m = m[None]
    ax = 1 if two_d else 0
    n = m.shape[ax]
    pieces = []
    for layer in part["box"]:
        lo, hi = layer * tile_a, min((layer + 1) * tile_a, n)
        pieces.append(m[:, lo:hi] if two_d else m[lo:hi])
    return np.ascontiguousarray(np.concatenate(pieces, axis=ax))


def node_rows(part: dict, tile_a: int, n: int, local: bool = True):
    """Node index ranges along the split axis of the rank's interior: local
    (within the box) or global."""
    b, e = part["interior"]
    if local:
        off = 0 if part["ghost_lo"] is None else min(tile_a, n)
        return off, off + min(part["hi"] * tile_a, n) - part["lo"] * tile_a
    return part["lo"] * tile_a, min(part["hi"] * tile_a, n)


class SlabSolver:
    """One rank's share of a domain-split run on its GPU.

    `comm` moves a layer's bytes between ranks: ``TorchDistComm`` (NCCL
    send/recv through torch.distributed) or, for several ranks driven from one
    process, ``LocalComm``.  Periodic flags apply to the global geometry; the
    split axis's flag decides whether the end slabs exchange with each other.
    """

    def __init__(self, mask, lattice, tile_a, periodic, tau, force, rank, world, comm, rho0=1.0,
                 model=lbm.LBM_QUASI_COMPRESSIBLE, arith=lbm.LBM_ARITH_AUTO, device="cuda"):
        m = np.asarray(mask, np.uint8)
        if m.ndim == 2:
            m = m[None]
        self.lattice, self.tile_a, self.rank, self.world = lattice, tile_a, rank, world
        ax = 2 if lattice == lbm.LBM_D3Q19 else 1      # index of the split axis in (x, y, z)
        n = split_axis_len(m, lattice)
        if periodic[ax] and n % tile_a:
            raise ValueError("a periodic split axis must be a multiple of the tile edge")
        n_layers = -(-n // tile_a)
        self.n_nodes_axis = n
        self.parts = plan(n_layers, world, bool(periodic[ax]))
        self.part = self.parts[rank]
        self.box = box_mask(m, lattice, tile_a, self.part)
        per = list(periodic)
        if world > 1:
            per[ax] = 0  # the box's split-axis ends are ghost layers (or the domain's walls)
        self.solver = lbm.Solver(self.box, lattice, tile_a, tuple(per), tau, force, rho0=rho0, model=model,
                                 arith=arith, device=device)
        self.comm = comm
        lib = lbm.library()
        self._ranges = {}
        nl = len(self.part["box"])
        for layer in range(nl):
            off, nb = ctypes.c_size_t(), ctypes.c_size_t()
            lbm._check(lib.lbm_layer_range(self.solver.ctx, layer, layer + 1, ctypes.byref(off), ctypes.byref(nb)))
            self._ranges[layer] = (off.value, nb.value)
        self.n_fluid_interior = int(self.interior_mask().sum())
        if comm is not None:
            comm.register(self)

    # -- geometry of the rank's share --------------------------------------------
    def interior_mask(self):
        lo, hi = node_rows(self.part, self.tile_a, self.n_nodes_axis)
        return self.box[lo:hi] if self.lattice == lbm.LBM_D3Q19 else self.box[:, lo:hi]

    def recv_list(self):
        return self.part["recv"]

    def layer_bytes(self, local_layer):
        """(offset, length) of a box layer in a PDF copy."""
        return self._ranges[local_layer]

    def current_copy(self):
        """The torch uint8 buffer that holds the current post-collision state."""
        return self.solver.pdf[lbm.library().lbm_current_copy(self.solver.ctx)]

    # -- stepping ------------------------------------------------------------------
    def step(self, n=1):
        for _ in range(n):
            self.solver.step(1)
            if self.world > 1:
                self.comm.exchange(self)

    def stats(self, residual=False, all_reduce=None):
        """Interior statistics of this rank, summed over the ranks by
        `all_reduce(list of 7 floats) -> list` when given."""
        st = lbm.lbm_stats()
        b, e = self.part["interior"]
        rc = lbm.library().lbm_moments_layers(self.solver.ctx, b, e, ctypes.byref(st),
                                               lbm.LBM_STATS_RESIDUAL if residual else 0, self.solver._s())
        if rc not in (lbm.LBM_OK, -5):
            lbm._check(rc)
        v = [st.mass, st.momentum[0], st.momentum[1], st.momentum[2], st.u2, st.du2, float(st.n_fluid)]
        if all_reduce is not None:
            v = all_reduce(v)
        res = float(np.sqrt(v[5] / v[4])) if residual and v[4] > 0 else float("inf")
        return {"mass": v[0], "momentum": v[1:4], "u2": v[4], "du2": v[5], "n_fluid": int(v[6]),
                "residual": res}

    def export_interior(self):
        """Dense FP64 post-collision PDFs of the rank's interior [q][z][y][x]."""
        full = self.solver.export_pdfs()
        lo, hi = node_rows(self.part, self.tile_a, self.n_nodes_axis)
        return full[:, lo:hi] if self.lattice == lbm.LBM_D3Q19 else full[:, :, lo:hi]

    def close(self):
        self.solver.close()


class TorchDistComm:
    """Ghost-layer exchange over torch.distributed (NCCL on GPUs): each step,
    every send and receive of the rank posted together (batch_isend_irecv)
    into the receiver's own PDF buffer."""

    def __init__(self, dist):
        self.dist = dist

    def register(self, s):
        pass

    def exchange(self, s):
        buf = s.current_copy()
        ops = []
        for peer, layer, g in s.part["send"]:
            off, nb = s.layer_bytes(layer)
            ops.append(self.dist.P2POp(self.dist.isend, buf[off:off + nb], peer, tag=g))
        for peer, layer, g in s.part["recv"]:
            off, nb = s.layer_bytes(layer)
            ops.append(self.dist.P2POp(self.dist.irecv, buf[off:off + nb], peer, tag=g))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()


class LocalComm:
    """The same exchange between ranks held by one process (one GPU): after
    every rank has stepped, each ghost layer is copied from the neighbour's
    interior layer with a device-to-device copy.  Step through ``step_all``
    (a rank stepping alone would run ahead of the others)."""

    def __init__(self):
        self.ranks = {}

    def register(self, s):
        self.ranks[s.rank] = s

    def exchange(self, s):
        raise RuntimeError("ranks of one process step together: use LocalComm.step_all")

    def _copy_ghosts(self):
        for r, me in self.ranks.items():
            dst = me.current_copy()
            for peer, layer, g in me.recv_list():
                other = self.ranks[peer]
                src_local = other.part["box"].index(g, other.part["interior"][0], other.part["interior"][1])
                so, snb = other.layer_bytes(src_local)
                do, dnb = me.layer_bytes(layer)
                if snb != dnb:
                    raise RuntimeError(f"layer {g}: {snb} bytes on rank {peer}, {dnb} on rank {r}")
                dst[do:do + dnb].copy_(other.current_copy()[so:so + snb])

    def step_all(self, n=1):
        """Step every rank n times, exchanging ghost layers after each step."""
        ranks = [self.ranks[r] for r in sorted(self.ranks)]
        for _ in range(n):
            for s in ranks:
                s.solver.step(1)
            if len(ranks) > 1:
                self._copy_ghosts()
