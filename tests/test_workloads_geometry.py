"""The seeded geometry inputs: each layout satisfies the rules of the convective outflow and the
inlet table (checked by the oracle's Geometry), and the emulsion generator carries the widths
and velocities Sec. V lists."""
import numpy as np
import pytest

import nfe_workloads as W
from oracle import boundaries as B
from oracle import lbm


@pytest.mark.parametrize("make", [lambda: W.open_channel_2d(), lambda: W.open_channel_2d(outflow=False),
                                  lambda: W.emulsion_2d(), lambda: W.porous_channel_2d(nx=256, ny=64),
                                  lambda: W.pals_2d()])
def test_layouts_are_valid_geometries(make):
    p = make()
    g = p["geometry"]
    prm = lbm.Params(p)
    geo = B.Geometry(prm, g["node"], g["inlets"], g["outflow"])
    assert np.allclose(g["inlets"][:, 2:].sum(axis=1), 1.0)
    assert np.allclose(p["C0"].sum(axis=0), 1.0)
    assert geo.fluid.sum() > 0.5 * geo.fluid.size or p["name"].startswith("emulsion")
    assert p["C0"].min() >= 0.0


def test_emulsion_generator_dimensions():
    p = W.emulsion_2d()
    node = p["geometry"]["node"][0]
    tab = p["geometry"]["inlets"]
    assert node.shape == (140, 600)
    widths = [int((node == W.INLET0 + j).sum()) for j in range(6)]
    assert widths == [10, 10, 8, 8, 51, 51]
    # fluids 3 and 4 enter at 0.003 along x, fluid 2 at 0.0045 and fluid 1 at 0.0098 across
    assert np.allclose(tab[:, 0], [0.003, 0.003, 0, 0, 0, 0])
    assert np.allclose(np.abs(tab[:, 1]), [0, 0, 0.0045, 0.0045, 0.0098, 0.0098])
    assert [int(np.argmax(r[2:])) for r in tab] == [2, 3, 1, 1, 0, 0]
    # inlet channels begin 55 sites from the bottom and top edges; the last channel is 110 high
    rows3 = np.nonzero(node[:, 0] == W.INLET0)[0]
    rows4 = np.nonzero(node[:, 0] == W.INLET0 + 1)[0]
    assert rows3.min() == 55 and rows4.max() == 140 - 55 - 1
    assert int((node[:, -1] == W.FLUID).sum()) == 110
