"""GPU parity of point sources (Sec. 4.2, Eq. SourceRho) against the oracle's
point_source, on a jittered 2^3 Kuhn cube with per-tet damping and boundary
reflection 0.8:

- the collapsed Gauss rule at order 48 against the oracle at the same order
  (the same rule: only rounding differs), for a source inside a tet, on an
  interior face, on an interior edge and at an interior vertex (24 tets);
- a source in a tet at the cube's corner, some of whose faces reflect;
- the default split polar rule against the oracle at order 128 (converged to
  ~1e-14 of the largest coefficient for these points);
- a source close to a face, where the flat rule loses digits: with mu = 0
  each face's (0,0) coefficient is the solid angle (Van Oosterom-Strackee)
  over pi sqrt|F| (times the reflection coefficient on the boundary) and the
  four faces together hold the full sphere;
- several sources in one call give the single-source rows bit for bit;
- the solve of I - B with point sources as right-hand sides against the
  dense solve of the GPU's own blocks;
- a source outside the mesh and a non-finite position are rejected."""
import numpy as np
import pytest

from gpu_helpers import need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu

REFL = 0.8


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


@pytest.fixture(scope="module")
def setup(D):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    mesh = D.Mesh(m.verts, m.tets, refl=REFL)
    mu = np.random.default_rng(3).uniform(0.1, 0.5, m.n_tets)
    return m, mesh, mu


def _points(V, T):
    tv = V[T[20]]
    inner = lambda x: np.all((x > 1e-9) & (x < 1 - 1e-9))  # noqa: E731
    face = next(tv[[k for k in range(4) if k != l]].mean(axis=0) for l in range(4)
                if inner(tv[[k for k in range(4) if k != l]].mean(axis=0)))
    edge = next((tv[i] + tv[j]) / 2 for i in range(4) for j in range(i + 1, 4) if inner((tv[i] + tv[j]) / 2))
    vid = 1 + 3 * (1 + 3 * 1)
    return {"inside": tv.mean(axis=0), "face": face, "edge": edge, "vertex": V[vid],
            "corner": V[T[0]].mean(axis=0)}


def _solid_angle(r, a, b, c):
    A, B, C = a - r, b - r, c - r
    la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(C)
    num = abs(A @ np.cross(B, C))
    den = la * lb * lc + (A @ B) * lc + (A @ C) * lb + (B @ C) * la
    return 2.0 * np.arctan2(num, den)


@pytest.mark.parametrize("where", ["inside", "face", "edge", "vertex", "corner"])
@pytest.mark.parametrize("Np", [3, 8])
def test_point_source_matches_oracle(D, oracle_mod, setup, where, Np):
    import torch

    m, mesh, mu = setup
    r0 = _points(m.verts, m.tets)[where]
    mu_t = torch.tensor(mu, device="cuda")
    for nq, oq, tol in ((48, 48, 1e-12), (0, 128, 1e-11)):
        got = D.point_source(mesh, Np, r0, mu=mu_t, strength=1.7, nq=nq)[0].cpu().numpy()
        want = oracle_mod.point_source(m.verts, m.tets, r0, Np, mu, REFL, strength=1.7, nq=oq)
        live = np.abs(want).max(axis=1) > 0
        assert live.sum() >= {"inside": 4, "face": 6, "edge": 8, "vertex": 24, "corner": 4}[where]
        assert np.all(got[~live] == 0.0)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= tol, (nq, err)


def test_source_close_to_a_face_keeps_the_solid_angles(D, oracle_mod, setup):
    m, mesh, _ = setup
    V, T = m.verts, m.tets
    P = V[T[20]]
    lam = np.array([0.3, 0.3, 0.3999, 1e-4])  # 1e-4 of the height above face 3
    r0 = lam @ P
    a = D.point_source(mesh, 0, r0, mu=0.0, strength=1.0)[0].cpu().numpy()
    A = oracle_mod.face_areas(V, T)
    recv = mesh.recv()
    total = 0.0
    for l in range(4):
        row = 4 * 20 + l
        p = V[[T[20, (l + 1 + k) % 4] for k in range(3)]]
        wgt = REFL if recv[row] == row else 1.0  # a boundary face reflects its share
        assert a[recv[row], 0] == pytest.approx(wgt * _solid_angle(r0, *p) / (np.pi * np.sqrt(A[row])), rel=1e-12)
        total += np.sqrt(A[row]) * a[recv[row], 0] / wgt
    assert total == pytest.approx(4.0, rel=1e-12)


def test_batched_sources_equal_single_calls(D, setup):
    import torch

    m, mesh, mu = setup
    pts = np.stack(list(_points(m.verts, m.tets).values()))
    mu_t = torch.tensor(mu, device="cuda")
    both = D.point_source(mesh, 4, pts, mu=mu_t)
    for s in range(pts.shape[0]):
        assert torch.equal(both[s], D.point_source(mesh, 4, pts[s], mu=mu_t)[0])


def test_solve_with_point_sources(D, oracle_mod, setup):
    import torch

    m, mesh, mu = setup
    nt = m.n_tets
    Np = 2
    mu_t = torch.tensor(mu, device="cuda")
    op = D.Operator(mesh, Np, mu=mu_t, precision=D.F32)
    pts = np.stack([_points(m.verts, m.tets)[k] for k in ("inside", "vertex")])
    rho0 = D.point_source(mesh, Np, pts, mu=mu_t)
    rho, info = op.solve(rho0, tol=1e-11)
    assert info.resid <= 1e-11
    recv = mesh.recv()
    t, f, fp = oracle_mod.pair_list(nt)
    blocks = to_oracle_layout(op.blocks().double().cpu().numpy(), recv, nt)
    same = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks),
                               dest=recv[4 * t + fp].reshape(4 * nt, 3).astype(np.int64))
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    for r in range(2):
        want = np.linalg.solve(M, rho0[r].cpu().numpy().ravel())
        assert np.linalg.norm(rho[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want)


def test_bad_positions_are_rejected(D, setup):
    m, mesh, _ = setup
    with pytest.raises(D.DFMError):
        D.point_source(mesh, 2, np.array([2.0, 0.5, 0.5]))  # outside the unit cube
    with pytest.raises(D.DFMError):
        D.point_source(mesh, 2, np.array([np.nan, 0.5, 0.5]))
    with pytest.raises(D.DFMError):
        D.point_source(mesh, 2, np.array([0.5, 0.5, 0.5]), nq=1)
