"""Parity at the full benchmark size: the channel at nz = 37 (314,389
patches, 2.6M fine nodes, BF16 network 228-1024x4-81, FP32 fields) run
through the same entry points and launch configuration as bench.py, checked
on sampled patches against the FP64 oracle.

The oracle cannot run the whole mesh, but every quantity up to the corrected
right-hand side at a patch's nodes depends only on the coarse cells within
two vertex rings of that patch: the residual at a fine node on the fine
cells around it, the network row of a patch on the residual at its nodes,
the extension at a node on the rows of the patches containing it, and the
rhs at a node on the extension around it.  So for each sampled patch the
oracle runs its whole hot-path step on that two-ring sub-mesh (exterior
vertices that are interior in the full mesh get the do-nothing kind, which
adds no term) and the results are compared at the patch; fine nodes of the
sub-mesh are matched to the full mesh by position."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_util import TOL  # noqa: E402
from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import dnnmg as odnnmg, mesh as omesh  # noqa: E402

NZ, DT, THETA = 37, 0.005, 0.5
WIDTHS = (228, 1024, 1024, 1024, 1024, 81)


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m = I.channel_mesh(NZ, seed=0)
    nu = m["meta"]["D"] / 200.0
    stream = torch.cuda.Stream()
    p = PatchPath(m, nu, DT, THETA, "bf16", stream=stream)
    Ws, ss, ts = I.network_weights(WIDTHS, seed=0)
    p.set_network(WIDTHS, Ws, ss, ts, skip=True)
    nc, nf = p.n_patches, p.n_fine
    xc_h = I.coarse_state(m, seed=0).astype(np.float32)
    F_h = I.fine_rhs(nf, seed=0, scale=(1 / DT) * 0.42 / (8 * nc)).astype(np.float32)
    with torch.cuda.stream(stream):
        xc, F = p.to_device(xc_h), p.to_device(F_h)
        r = p.residual(xc, F)
        X = p.local_restrict(xc, r)
        Y = p.network(X, nc)
        d = p.extend(Y)
        bf, _ = p.rhs_restrict(xc, d)
    torch.cuda.synchronize()
    capi.dnnmg_sync(p.ctx, 10_000_000)
    out = dict(m=m, nu=nu, net=(Ws, ss, ts), xc=xc_h.astype(np.float64), F=F_h.astype(np.float64),
               r=r.cpu().numpy(), X=X.float().cpu().numpy(), Y=Y.cpu().numpy(), d=d.cpu().numpy(),
               bf=bf.cpu().numpy(), pm=p.mesh_data(capi.PATCH_MAP), fxyz=p.mesh_data(capi.FINE_XYZ), nc=nc)
    p.close()
    return out


def _samples(m, nc):
    cen = m["xyz"][m["cells"]].mean(axis=1)
    meta = m["meta"]
    dist = np.hypot(cen[:, 0] - meta["cx"], cen[:, 1] - meta["cy"])
    picks = [int(np.argmin(dist)),                 # at the cylinder
             int(np.argmin(cen[:, 0])),            # at the inflow
             int(np.argmax(cen[:, 0])),            # at the outflow
             int(np.argmin(cen[:, 2] + np.abs(cen[:, 0] - 0.5 * cen[:, 0].max())))]   # at a wall, mid-channel
    u = I.splitmix_uniform(77, 8)
    picks += [int(x * nc) for x in u]              # seeded interior picks
    return picks


def _sub_mesh(m, P, v2c):
    cells = m["cells"]
    ring = [P]
    seen = {P}
    for _ in range(2):
        nxt = []
        for c in ring:
            for v in cells[c]:
                for c2 in v2c[v]:
                    if c2 not in seen:
                        seen.add(c2)
                        nxt.append(c2)
        ring = ring + nxt
    sub = np.array(ring)                          # the patch first, then its two rings
    verts, inv = np.unique(cells[sub].ravel(), return_inverse=True)
    csub = inv.reshape(-1, 8)
    bc = m["vertex_bc"][verts].copy()
    counts = {}
    for c in csub:
        for f in omesh.LOCAL_FACES:
            key = tuple(sorted(int(c[k]) for k in f))
            counts[key] = counts.get(key, 0) + 1
    for key, cnt in counts.items():
        if cnt == 1:
            for v in key:
                if bc[v] == 0:
                    bc[v] = 3
    ring1 = set()
    for v in cells[P]:
        ring1.update(v2c[v])
    ring1_local = [i for i, c in enumerate(sub) if c in ring1]
    return sub, verts, csub, bc, ring1_local


def test_sampled_patches_match_the_oracle(full):
    from scipy.spatial import cKDTree
    m, nc = full["m"], full["nc"]
    cells = m["cells"]
    v2c = [[] for _ in range(m["xyz"].shape[0])]
    for c in range(nc):
        for v in cells[c]:
            v2c[v].append(c)
    tree = cKDTree(full["fxyz"])
    Ws, ss, ts = full["net"]
    prm = dict(m=1.0 / DT, theta=THETA, nu=full["nu"], alpha0=0.02, delta0=0.1)
    tol = TOL["bf16"]
    picks = _samples(m, nc)
    checked = 0
    for P in picks:
        sub, verts, csub, bc, ring1 = _sub_mesh(m, P, v2c)
        h = omesh.Hierarchy(m["xyz"][verts], csub, bc)
        dist, gidx = tree.query(h.xyz_f)
        assert dist.max() < 1e-9
        o = odnnmg.hot_path_step(h, (Ws, ss, ts, True), full["xc"][verts], full["F"][gidx], prm)
        nodes_sub = h.patch_map[0]
        nodes = full["pm"][P]
        assert np.array_equal(gidx[nodes_sub], nodes)          # the same 27 nodes
        # the input row: x~ and r within bf16 rounding
        Xo, Xg = o["X"][0], full["X"][P, :228]
        xs = np.abs(o["X"][ring1]).max()
        assert np.all(np.abs(Xg - Xo) <= 2.0 ** -8 * np.abs(Xo) + 1e-5 * xs), P
        # the FP32 residual at the patch nodes
        Fs = full["F"][gidx]
        scale = np.abs(Fs).max() + np.abs(Fs - o["r"]).max()
        assert np.abs(full["r"][nodes] - o["r"][nodes_sub]).max() <= TOL["fp32"] * scale, P
        # the network row (per-patch norm, floored by the neighbourhood's median)
        nrm = np.linalg.norm(o["Y"][ring1], axis=1)
        den = max(np.linalg.norm(o["Y"][0]), 0.1 * float(np.median(nrm)))
        assert np.linalg.norm(full["Y"][P] - o["Y"][0]) <= tol * den, P
        # extension and corrected rhs at the patch nodes
        dmax = np.abs(o["d"][nodes_sub]).max()
        assert np.abs(full["d"][nodes] - o["d"][nodes_sub]).max() <= tol * dmax + 1e-30, P
        bmax = np.abs(o["b_fine"][nodes_sub]).max()
        assert np.abs(full["bf"][nodes] - o["b_fine"][nodes_sub]).max() <= tol * bmax + 1e-30, P
        checked += 1
    assert checked == len(picks) == 12
