"""Host-side logic of the accessor (Sec. 3, "How to use the implementation?"): how an index is
split into the channel entry and the spatial entries, slices read as linspace, and the output
shapes of point and volume queries; the plan's default M2L form.  No GPU."""
import numpy as np
import pytest
import torch

from paper_2111_00110_gb300.accessor import WIDTH, grid_shape, parse_key, point_shape, select_channels


def test_slice_is_linspace_with_domain_defaults():
    chan, coords, scalar = parse_key((0, slice(0.25, 0.75, 3), slice(None, None, 5), 0.5), 3, 0.0, 1.0)
    assert chan == 0
    assert np.allclose(coords[0].numpy(), [0.25, 0.5, 0.75])
    assert np.allclose(coords[1].numpy(), np.linspace(0.0, 1.0, 5))
    assert coords[2].dim() == 0 and scalar == [False, False, True]


def test_channel_entry_forms():
    for key, chan in (((0.1, 0.2, 0.3), Ellipsis), ((Ellipsis, 0.1, 0.2, 0.3), Ellipsis),
                      ((slice(0, 2), 0.1, 0.2, 0.3), slice(0, 2)), (([0, 2], 0.1, 0.2, 0.3), [0, 2])):
        assert parse_key(key, 3, 0.0, 1.0)[0] == chan
    with pytest.raises(IndexError):
        parse_key((0.1, 0.2), 3, 0.0, 1.0)
    with pytest.raises(IndexError):
        parse_key((0, 0.1, Ellipsis, 0.3), 3, 0.0, 1.0)
    with pytest.raises(IndexError):
        parse_key((slice(0.0, 1.0), 0.2, 0.3), 3, 0.0, 1.0)   # no count


def test_point_and_volume_shapes():
    _, c, _ = parse_key((slice(0, 1, 4), slice(0, 1, 4), 0.0), 3, 0.0, 1.0)
    assert point_shape(c) == (4,)
    assert grid_shape(c) == (4, 4, 1)
    _, c, _ = parse_key((slice(0, 1, 128), slice(0, 1, 64), 0.0), 3, 0.0, 1.0)
    assert grid_shape(c) == (128, 64, 1)
    _, c, _ = parse_key((0.1, 0.2, 0.3), 3, 0.0, 1.0)
    assert point_shape(c) == ()
    _, c, _ = parse_key((torch.rand(6), torch.rand(6)), 2, 0.0, 1.0)
    assert point_shape(c) == (6,)
    assert WIDTH["partials"](3) == 3 and WIDTH["partials2"](3) == 6 and WIDTH["partials2"](2) == 3


def test_channel_selection():
    out = torch.arange(24.0).reshape(4, 6)
    assert select_channels(out, Ellipsis).shape == (4, 6)
    assert select_channels(out, 1).shape == (6,)
    assert select_channels(out, slice(1, 3)).shape == (2, 6)
    assert torch.equal(select_channels(out, [3, 0]), out[[3, 0]])


def test_plan_m2l_auto_resolution():
    """A plan's default M2L form: the separable line passes where they apply (the Gaussian in 3D
    with Taylor operators), plain FP32 otherwise; an explicit form is kept."""
    from paper_2111_00110_gb300.transform import resolve_m2l
    assert resolve_m2l("auto", 3, "gaussian", False) == "separable"
    assert resolve_m2l("auto", 2, "gaussian", False) == "fp32"
    assert resolve_m2l("auto", 3, "poly", False) == "fp32"
    assert resolve_m2l("auto", 3, "gaussian", True) == "fp32"
    for form in ("fp32", "tf32", "bf16", "tf32x3", "bf16x3", "separable"):
        assert resolve_m2l(form, 3, "gaussian", False) == form
