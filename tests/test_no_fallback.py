"""The Python front end has no CPU path (no GPU needed): without libstp.so every entry point
raises, and tensors that are not on a CUDA device are refused before any call is made."""
import numpy as np
import pytest
import torch

from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import inputs as I
from paper_2402_00525_gb300 import renderer as R


def test_missing_library_raises_everywhere(monkeypatch, tmp_path):
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "libstp.so"))
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        N.lib()
    cam = I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 32, 32, 60.0)
    with pytest.raises(RuntimeError, match="not built"):
        R.Renderer(100, [cam], I.RenderParams(), device="cpu")


def test_host_tensors_are_refused():
    g = R.scene_to_device(I.uniform_scene(64, 1), device="cpu")
    with pytest.raises(ValueError, match="CUDA"):
        R.gaussians_struct(g)
    g = {k: v for k, v in g.items()}
    g["means"] = torch.from_numpy(np.zeros((64, 3), np.float64))
    with pytest.raises(ValueError):
        R.gaussians_struct(g)
