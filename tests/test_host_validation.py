"""Argument checks of rad_init and rad_pic_init, which run on the host before
any device call: every malformed configuration is RAD_EINVAL on any machine,
and (without a GPU) a well-formed one gets past them and stops at the device
(RAD_ECUDA from the device query, RAD_PIC_ENOMEM from the first allocation)."""
import math

import numpy as np
import pytest

EINVAL = -1


def _no_gpu():
    torch = pytest.importorskip("torch")
    return not torch.cuda.is_available()


def _radiation(**kw):
    from paper_1003_1140_gb300 import rad as R
    a = dict(dirs=np.array([[0.0, 1.0, 0.0]]), grids=[np.linspace(1.0, 2.0, 4)], dt=0.1,
             species=[(8, -1.0)], windows=[(0, 4, 1, 0)])
    a.update(kw)
    return R.Radiation(a["dirs"], a["grids"], a["dt"], a["species"], a["windows"],
                       mode=a.get("mode", 0), precision=a.get("precision", 1),
                       box_L=a.get("box_L", 0.0))


@pytest.mark.parametrize("bad", [
    {"dirs": np.zeros((0, 3))},                       # no direction
    {"grids": [np.array([])]},                        # empty frequency grid
    {"grids": [np.array([1.0, math.nan])]},           # non-finite frequency
    {"dt": 0.0}, {"dt": -0.1}, {"dt": math.nan}, {"dt": math.inf},
    {"species": [(-1, -1.0)]},                        # negative count
    {"species": [(4, math.nan)]},                     # non-finite charge
    {"species": [(4, -1.0)] * 33},                    # more species than supported
    {"windows": [(5, 3, 1, 0)]},                      # s1 < s0
    {"windows": [(-1, 3, 1, 0)]},                     # s0 < 0
    {"windows": [(0, 3, 1, 1)]},                      # grid index out of range
    {"windows": [(0, 3, 2, 0)]},                      # species bit beyond the species
    {"windows": [(0, 3, 1, 0, [1])]},                 # direction index beyond the directions
    {"windows": [(0, 3, 1, 0, [0, -1])]},             # negative direction index
    {"windows": [(0, 3, 1, 0, [])]},                  # an empty direction set
    {"mode": 2}, {"precision": 2},
    {"box_L": -1.0}, {"box_L": math.nan}, {"box_L": math.inf},
])
def test_rad_init_rejects_malformed_configurations(bad):
    from paper_1003_1140_gb300 import rad as R
    with pytest.raises(R.RadError) as ei:
        _radiation(**bad)
    assert ei.value.code == EINVAL


def test_rad_init_accepts_a_wellformed_configuration_up_to_the_device():
    if not _no_gpu():
        pytest.skip("a GPU is present: the configuration would simply succeed")
    from paper_1003_1140_gb300 import rad as R
    with pytest.raises(R.RadError) as ei:
        _radiation(box_L=2.0, windows=[(0, 4, 1, 0), (2, 2, 1, 0), (1, 3, 1, 0, [0, 0])])
    assert ei.value.code == -3


def _pic(n=16, d=0.1, dt=0.05, species=((2, -1.0, 1.0, 1.0),), x="ok", u="ok"):
    from paper_1003_1140_gb300 import pic
    N = sum(int(s[0]) for s in species)
    xx = np.full((3, max(N, 1)), 0.5) if x == "ok" else x
    uu = np.zeros((3, max(N, 1))) if u == "ok" else u
    return pic.Pic(n, d, dt, list(species), xx, uu)


@pytest.mark.parametrize("bad", [
    {"n": 3}, {"n": 20000},                            # grid size
    {"d": 0.0}, {"d": math.nan}, {"d": math.inf},
    {"dt": 0.0}, {"dt": math.nan}, {"dt": math.inf},
    {"dt": 0.08},                                      # Courant: dt >= d / sqrt(2)
    {"species": ((-1, -1.0, 1.0, 1.0),)},              # negative count
    {"species": ((2, -1.0, 0.0, 1.0),)},               # zero mass
    {"species": ((2, math.nan, 1.0, 1.0),)},           # non-finite charge
    {"species": ((2, -1.0, 1.0, math.inf),)},          # non-finite weight
    {"species": ((1, -1.0, 1.0, 1.0),) * 9},           # more species than supported
    {"x": None}, {"u": None},                          # particles without a state
])
def test_rad_pic_init_rejects_malformed_configurations(bad):
    with pytest.raises(RuntimeError) as ei:
        _pic(**bad)
    assert "(-1)" in str(ei.value)


def test_rad_pic_init_accepts_a_wellformed_configuration_up_to_the_device():
    if not _no_gpu():
        pytest.skip("a GPU is present: the configuration would simply succeed")
    with pytest.raises(RuntimeError) as ei:
        _pic()
    assert "(-2)" in str(ei.value)
