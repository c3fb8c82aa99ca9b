"""What storing the distributions in a narrow format costs, measured on the
FP64 oracle.

Storage precision enters the step only through the stored state: the
distributions are rounded once per step when they are written, and every
operation on them runs in a wider type (FP32 arithmetic with FP64 W for FP32
storage; the same would hold for BF16 storage).  So the oracle, with its state
rounded to the storage format after every step (W, the tracked conserved
variables, stays FP64 as in the GPU path), carries exactly the storage error
of that format, free of any other rounding.  Against the unrounded oracle on
the 2D Kelvin-Helmholtz physics (32^2 velocities reduced to 16^2 here) and
the 3D shear physics:

* FP32 storage (24-bit significand) stays far inside the 1e-5 target on rho,
  u, T that the FP32 path is held to;
* BF16 storage (8-bit significand) misses it by orders of magnitude, which is
  why the path has no BF16 variant.

Each test prints the errors (run with -s)."""
import numpy as np
import pytest

from paper_2208_09132_gb300 import workloads as wl
from test_gpu_parity import rel_linf

TOL = 1e-5


def round_fp32(x):
    return x.astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even): the upper 16 bits of the
    FP32 encoding, after rounding FP64 to FP32 (both round to nearest even;
    double rounding cannot matter at the tolerances checked here)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_is_round_to_nearest_even():
    # exact bfloat16 values stay, halfway cases go to the even neighbour
    assert round_bf16(np.array([1.0, -2.5, 0.0]))[0] == 1.0
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9])
    assert list(round_bf16(x)) == [1.0, 1.0 + 4 * 2.0 ** -8, 1.0]
    r = np.random.default_rng(0).uniform(0.5, 2.0, 1000)
    assert np.all(np.abs(round_bf16(r) - r) <= 2.0 ** -8 * r)


def run(oracle_mod, cfg, f, steps, rounding):
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    if rounding is not None:
        g, b = o.distributions()
        o.set_state(rounding(g), rounding(b), o.conserved())
    for _ in range(steps):
        o.step(1)
        if rounding is not None:
            g, b = o.distributions()
            o.set_state(rounding(g), rounding(b), o.conserved())
    return o.moments()


@pytest.mark.parametrize("name,case,steps", [
    ("kh2d 24^2 x 16^2", lambda: wl.kelvin_helmholtz(n=24, nv=16, kn=1e-3), 100),
    ("shear3d 6^3 x 12^3", lambda: wl.shear3d(n=6, nv=12, kn=1e-2), 30),
])
def test_storage_rounding_error(oracle_mod, name, case, steps):
    cfg, f = case()
    ref = run(oracle_mod, cfg, f, steps, None)
    e32 = rel_linf(run(oracle_mod, cfg, f, steps, round_fp32), ref)
    e16 = rel_linf(run(oracle_mod, cfg, f, steps, round_bf16), ref)
    print(f"\n[storage] {name}, {steps} steps: rel Linf rho,u,T FP32 storage "
          f"{', '.join(f'{e:.1e}' for e in e32)}; BF16 storage {', '.join(f'{e:.1e}' for e in e16)}")
    assert np.all(e32 <= TOL / 10)
    assert np.max(e16) > 10 * TOL
