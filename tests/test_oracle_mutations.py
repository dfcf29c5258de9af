"""Mutation test of the oracle's pins: each planted mistake below is compiled
into a second copy of the oracle's C code (-DORC_MUTATE=k), swapped in for the
real one, and at least one pin must fail on it.  The mistakes are the kinds a
reader checks the oracle against the paper for: a sin/cos mix-up in the
Zernike polynomials, a dropped normalisation factor, the wrong face frame for
the receiving face, a halved damping exponent, a transposed operator, an
unnormalised tangent axis, a missing clip of the integration triangle, a dropped
cosine in the interior density, swapped impedances in the transmission law,
an inverted Snell ratio, a reflection weighted like a transmission, and two in the
linear spatial basis (the receiving function read at the ray's start, a wrong mass matrix).  A second set plants mistakes in the oracle's
Python half (a reversed point-source ray, |T| for sqrt|T|, a dropped inverse
norm, a left-handed frame, a left-out reflection part) by rewriting one line of
the function's source.  Only the oracle is mutated, on the CPU."""
import ctypes
import os
import subprocess

import pytest

import test_oracle_blocks as blocks
import test_oracle_media as media
import test_oracle_p1 as p1
import test_oracle_solve as solve
import test_oracle_source as source
import test_oracle_zernike as zernike

MUTANTS = {
    1: "Zernike: cos instead of sin for m < 0",
    2: "inverse norm without eps_m",
    3: "receiving Zernike vector in the source face frame",
    4: "damping exponent halved",
    5: "transposed application applies B",
    6: "first tangent axis not normalised (e1 = second - first vertex)",
    7: "integration triangle not clipped to the source face",
    8: "interior density without the cosine",
    9: "impedances swapped in the transmission law",
    10: "inverted Snell ratio for the transmitted direction",
    11: "interface reflection weighted by lambda_t instead of 1 - lambda_t",
    12: "linear spatial basis: receiving function read at the source point",
    13: "linear spatial basis: Gram-Schmidt with a wrong mass matrix",
}


def _pins(O):
    """Cheap pins (no Monte Carlo except for the Snell mutant's own check)."""
    yield lambda: zernike.test_orthogonality(O)
    yield lambda: zernike.test_closed_form_matches_paper_recursion(O, 4)
    yield lambda: blocks.test_regular_tet_view_factor(O)
    yield lambda: blocks.test_reciprocity_single_tet(O, 0.8)
    yield lambda: blocks.test_conservation_weighted_column_sums(O)
    yield lambda: solve.test_interior_kernel_solid_angles(O)
    yield lambda: solve.test_adjoint_identity_and_fd(O)
    yield lambda: source.test_textbook_low_orders_on_a_known_frame(O)
    yield lambda: source.test_rotation_about_the_normal(O)
    yield lambda: media.test_transmission_law(O)


def _build_mutant(O, k, outdir):
    src = os.path.join(os.path.dirname(O.build()), "..", "dfm_oracle.c")
    so = os.path.join(outdir, f"liboracle_mut{k}.so")
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", f"-DORC_MUTATE={k}", "-o",
                           so, os.path.abspath(src), "-lm"])
    L = ctypes.CDLL(so)
    os.remove(so)  # the loaded copy stays mapped
    L.orc_blocks.restype = ctypes.c_int
    L.orc_mc_block.restype = ctypes.c_int
    L.orc_blocks_p1.restype = ctypes.c_int
    L.orc_mc_block_p1.restype = ctypes.c_int
    L.orc_region_cos_measure.restype = ctypes.c_double
    L.orc_transmission.restype = ctypes.c_double
    L.orc_transmission.argtypes = [ctypes.c_double] * 4
    return L


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_a_pin_fails_on_each_planted_mistake(oracle_mod, k):
    import oracle.oracle as core

    real = core.lib()
    outdir = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(outdir, exist_ok=True)
    core._lib = _build_mutant(oracle_mod, k, outdir)
    failed = []
    try:
        pins = list(_pins(oracle_mod))
        if k == 10:
            pins = [lambda: media.test_monte_carlo_across_an_interface(oracle_mod, 1)]
        if k == 11:
            pins = [lambda: media.test_conservation_with_unequal_media(oracle_mod)]
        if k == 12:
            pins = [lambda: p1.test_reciprocity_linear_basis(oracle_mod, 0.8)]
        if k == 13:
            pins = [lambda: p1.test_linear_basis_is_orthonormal(oracle_mod)]
        for pin in pins:
            try:
                pin()
            except AssertionError:
                failed.append(pin)
                break
    finally:
        core._lib = real
    assert failed, f"no pin caught mutant {k}: {MUTANTS[k]}"


def test_the_real_oracle_passes_the_same_pins(oracle_mod):
    for pin in _pins(oracle_mod):
        pin()


# Mistakes planted in the oracle's Python half: (function, original text, planted text, pin).
PY_MUTANTS = {
    "point source: ray direction reversed": (
        "point_source", "Z = zernike(Np, (uv @ e1[rec]).reshape(-1), (uv @ e2[rec]).reshape(-1))",
        "Z = zernike(Np, (-uv @ e1[rec]).reshape(-1), (-uv @ e2[rec]).reshape(-1))",
        lambda O: __import__("test_oracle_point_source").test_rays_arrive_pointing_away_from_the_source(O)),
    "isotropic source: |T| instead of sqrt|T|": (
        "source_vector", "x[int(r), 0] += wt * np.sqrt(area[int(r)])", "x[int(r), 0] += wt * area[int(r)]",
        lambda O: source.test_tet_density_of_an_isotropic_face_is_its_solid_angle(O)),
    "directed source: inverse norm dropped": (
        "source_directed", "out[s, r, :nz] = inv * zernike(Np, p[0], p[1])[0] * np.sqrt(area[r])",
        "out[s, r, :nz] = zernike(Np, p[0], p[1])[0] * np.sqrt(area[r])",
        lambda O: source.test_normal_incidence_closed_form(O)),
    "face frames: left-handed": (
        "face_frames", "e1[f::4], nn[f::4], e2[f::4] = u, n, np.cross(n, u)",
        "e1[f::4], nn[f::4], e2[f::4] = u, n, np.cross(u, n)",
        lambda O: source.test_textbook_low_orders_on_a_known_frame(O)),
    "application: interface reflections left out": (
        "apply", "if op.rblocks is not None:", "if False:",
        lambda O: media.test_conservation_with_unequal_media(O)),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_a_pin_fails_on_each_planted_python_mistake(oracle_mod, name):
    import inspect

    import oracle.oracle as core

    fname, old, new, pin = PY_MUTANTS[name]
    real = getattr(core, fname)
    src = inspect.getsource(real)
    assert old in src, f"{fname}: the text to mutate is gone"
    ns = dict(core.__dict__)
    exec(compile(src.replace(old, new), core.__file__, "exec"), ns)
    setattr(core, fname, ns[fname])
    setattr(oracle_mod, fname, ns[fname])
    try:
        with pytest.raises(AssertionError):
            pin(oracle_mod)
    finally:
        setattr(core, fname, real)
        setattr(oracle_mod, fname, real)
