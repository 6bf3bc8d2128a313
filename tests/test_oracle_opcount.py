"""The oracle's floating-point work per particle-step, counted by compiling it with an
op-counting scalar (oracle/opcount.cpp): the figure the push kernel's executed count is set
against (the kernel's 1049 flop per particle-step vs the oracle's plain definitions, which
form every term of Eqs. 1-2 separately from full Jacobians and 8-corner weights)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import AU
from paper_2403_06706_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "oracle", "opcount.cpp")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_oracle_flop_per_particle_step(tmp_path):
    exe = str(tmp_path / "opcount")
    subprocess.run(["g++", "-std=c++17", "-O2", "-o", exe, SRC], check=True, capture_output=True)
    w = synth.WindSpec(64, 32, 64, eps=0.1, n_modes=8)
    nodes = synth.wind_grid(w, dtype=np.float32)
    path = str(tmp_path / "nodes.f32")
    nodes.tofile(path)
    out = subprocess.run([exe, path, "64", "32", "64", repr(w.r_min_au * AU), repr(w.r_max_au * AU), "400", "64"],
                         check=True, capture_output=True, text=True).stdout.split()
    flop, collisions = float(out[0]), int(out[1])
    print("oracle flop per particle-step", flop, "collisions", collisions)
    # two field evaluations per step dominate; collisions and rebirths add a few restarts
    assert 3300 < flop < 3500
