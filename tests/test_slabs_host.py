"""Host side of the z-slab decomposition (no GPU): the slab bounds, the plane
slot ranges of the packed layout, and the face-exchange protocol of the
multi-process path, run as gloo ranks on the CPU.

The protocol test gives every rank its slab's state as a host array in the
packed layout, where the value of (direction i, slot of cell y) encodes the
box index of y and i.  The ranks exchange their faces with the same
exchange_faces the GPU path uses; afterwards the halo plane of every slab must
hold, at the pull source y - c_i of each of its interior cells next to the
face and each direction i with c_z pointing into the slab, the code of that
same cell and direction in the unsharded box, and nothing else may change."""

import itertools
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem
from paper_2402_10809_gb300 import lbm, slabs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def spans(flags):
    """Per row (y + ny z): first x of its non-solid span and its length."""
    nz, ny, nx = flags.shape
    rows = ((flags >= 1) & (flags <= 3)).reshape(nz * ny, nx)
    has = rows.any(1)
    lo = np.where(has, rows.argmax(1), 0)
    hi = np.where(has, nx - 1 - rows[:, ::-1].argmax(1), -1)
    return lo, np.where(has, hi - lo + 1, 0)


@pytest.mark.parametrize("n,nslabs", [(64, 2), (64, 3), (64, 4), (128, 3)])
def test_slab_bounds_balance_packed_slots(n, nslabs):
    prob = aneurysm_problem(n)
    b = slabs.slab_bounds(prob, nslabs)
    assert b[0] == 0 and b[-1] == n and all(b[k] < b[k + 1] for k in range(nslabs))
    _, ext = spans(prob.flags)
    per_plane = ext.reshape(n, n).sum(1)
    share = [per_plane[b[k]:b[k + 1]].sum() for k in range(nslabs)]
    assert abs(max(share) - per_plane.sum() / nslabs) <= per_plane.max()


def test_plane_slots_are_the_packed_ranges():
    prob = aneurysm_problem(64)
    f = np.ascontiguousarray(prob.flags)
    g = lbm.make_grid(prob.dims, 27, "f32", (0, 0, 0))
    _, ext = spans(f)
    per_plane = ext.reshape(64, 64).sum(1)
    first = np.concatenate([[0], np.cumsum(per_plane)])
    for z in range(64):
        assert lbm.lbm_plane_slots(g, f.ctypes.data, z) == (int(first[z]), int(per_plane[z]))
    assert first[-1] == lbm.lbm_list_length(g, f.ctypes.data)


def test_periodic_z_box_is_not_sharded():
    with pytest.raises(ValueError):
        slabs.slab_bounds(periodic_box_problem(8, 8, 8), 2)


WORKER = r"""
import itertools, json, os, sys
sys.path.insert(0, os.environ["REPO"])
import numpy as np, torch
import torch.distributed as dist
sys.path.insert(0, os.path.join(os.environ["REPO"], "tests"))
from test_slabs_host import spans
from lbm_inputs import aneurysm_problem
from paper_2402_10809_gb300 import lbm, slabs

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
n, q = int(os.environ["BOX"]), 27
prob = aneurysm_problem(n, small=False)
C = [c for c in itertools.product((-1, 0, 1), repeat=3)]  # (cz, cy, cx) of the 27 directions
cz = np.array([c[0] for c in C])
b = slabs.slab_bounds(prob, world)
z0, z1 = b[rank], b[rank + 1]
sub, h0, h1 = slabs.slab_problem(prob, z0, z1)
f = sub.flags
nzs, ny, nx = f.shape
lo, ext = spans(f)
base = np.concatenate([[0], np.cumsum(ext)])[:-1] - lo      # slot of (x, row) = base[row] + x
nst = int(ext.sum())
fluid = (f >= 1) & (f <= 3)
state = np.full((q, nst), -1, np.int64)
zz, yy, xx = np.nonzero(fluid)
rows = yy + ny * zz
slot = base[rows] + xx
gidx = xx + nx * (yy + ny * (zz + z0 - h0))                  # box index of the cell
inner = (zz >= h0) & (zz < nzs - h1)
for i in range(q):
    state[i, slot[inner]] = gidx[inner] * q + i
grid = lbm.make_grid((nx, ny, nzs), q, "f32", (0, 0, 0))
fc = np.ascontiguousarray(f)
def plane_range(z):
    a, c = lbm.lbm_plane_slots(grid, fc.ctypes.data, z)
    return a, a + c
def dirs(s):
    return [i for i in range(q) if cz[i] == s]
def face(side, pack):
    # side 0: send plane h0 with c_z = -1, receive plane 0 with c_z = +1; side 1 mirrored
    if side == 0:
        return (plane_range(h0), dirs(-1)) if pack else (plane_range(0), dirs(+1))
    return (plane_range(nzs - 1 - h1), dirs(+1)) if pack else (plane_range(nzs - 1), dirs(-1))
def pack(side, buf):
    (a, e), d = face(side, True)
    buf.copy_(torch.from_numpy(state[d, a:e].reshape(-1).astype(np.float64)))
def unpack(side, buf):
    (a, e), d = face(side, False)
    state[d, a:e] = buf.numpy().reshape(len(d), e - a).astype(np.int64)
send, recv = {}, {}
for side in (0, 1):
    if (h0, h1)[side]:
        (a, e), d = face(side, True)
        send[side] = torch.empty(len(d) * (e - a), dtype=torch.float64)
        recv[side] = torch.empty(slabs.face_message_elements(f, q, side, h0, h1), dtype=torch.float64)
before = state.copy()
slabs.exchange_faces(dist, rank, world, pack, unpack, send, recv)
# every pull across a face finds the unsharded box's value at its source
bad, checked = 0, 0
for zl, halo_z, s in ((h0, 0, +1), (nzs - 1 - h1, nzs - 1, -1)):
    if (h0 if s == +1 else h1) == 0:
        continue
    for i in dirs(s):
        cy, cx = C[i][1], C[i][2]
        ys, xs = np.nonzero(fluid[zl])
        for y, x in zip(ys, xs):
            sy, sx = y - cy, x - cx
            if not (0 <= sy < ny and 0 <= sx < nx) or not fluid[halo_z, sy, sx]:
                continue
            want = (sx + nx * (sy + ny * (halo_z + z0 - h0))) * q + i
            got = state[i, base[sy + ny * halo_z] + sx]
            checked += 1
            bad += int(got != want)
changed = np.argwhere(state != before)
zs_changed = set()
for i, sl in changed:
    r = int(np.searchsorted(base + lo + ext, sl, side="right"))
    zs_changed.add(r // ny)
print(json.dumps({"rank": rank, "checked": checked, "bad": bad, "planes_changed": sorted(zs_changed),
                  "halo_planes": [z for z, h in ((0, h0), (nzs - 1, h1)) if h]}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_face_exchange_protocol_on_gloo_ranks(world):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), REPO=ROOT, BOX="48", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    res = [p.communicate(timeout=300) + (p.returncode,) for p in procs]
    for o, e, rc in res:
        assert rc == 0, e[-3000:]
    out = [json.loads(o.strip().splitlines()[-1]) for o, _, _ in res]
    for d in out:
        assert d["bad"] == 0 and d["checked"] > 100, d
        assert d["planes_changed"] == d["halo_planes"], d  # only halo planes receive anything
