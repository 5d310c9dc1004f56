"""Host logic of bench.py that needs no GPU: argument defaults and the lookup of
the ncu DRAM traffic from the committed profile summaries."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _parse(argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench.parse()


def test_rayleigh_default_follows_the_dimension(monkeypatch):
    assert _parse([], monkeypatch).Ra == 1e8                      # 2-D cavity workload
    assert _parse(["--dim", "3", "--n", "256"], monkeypatch).Ra == 1e7   # 3-D cavity workload
    assert _parse(["--dim", "3", "--Ra", "1e5"], monkeypatch).Ra == 1e5


@pytest.fixture
def fake_tree(tmp_path, monkeypatch):
    """A repository root with stand-in kernel sources and a profiles folder."""
    csrc = tmp_path / "paper_2509_01099_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for dim in (2, 3):
        for name in bench.KERNEL_SOURCES[dim]:
            (csrc / name).write_text(f"// {name}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _summary(root, name, sha, traffic, nodes=None):
    lines = [f"# {name}", "", f"- source_sha256: `{sha}` (sources)",
             f"- traffic_bytes_per_launch: {traffic}"]
    if nodes is not None:
        lines.append(f"- nodes_per_launch: {nodes}")
    (root / "profiles" / name).write_text("\n".join(lines) + "\n")


def test_profile_traffic_exact_size(fake_tree):
    _summary(fake_tree, "step2d_fp32_tanh1024.md", bench.kernel_source_sha(2), 69809408)
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) == 69809408
    # another size: the summary does not state its node count, so nothing is scaled
    assert bench.profile_traffic(2, "fp32", "tanh", 4096) is None
    assert bench.profile_traffic(2, "bf16dev", "tanh", 1024) is None


def test_profile_traffic_scaled_by_stated_nodes(fake_tree):
    _summary(fake_tree, "step3d_fp32_tanh128.md", bench.kernel_source_sha(3), 1000,
             nodes=128 ** 3)
    assert bench.profile_traffic(3, "fp32", "tanh", 128) == 1000
    assert bench.profile_traffic(3, "fp32", "tanh", 256) == pytest.approx(8000)


def test_profile_traffic_ignores_a_stale_source_hash(fake_tree):
    _summary(fake_tree, "step2d_fp32_tanh1024.md", "0" * 64, 123)
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) is None
    # a kernel source edited after the capture also makes the summary stale
    _summary(fake_tree, "step2d_fp32_tanh1024.md", bench.kernel_source_sha(2), 123)
    src = fake_tree / "paper_2509_01099_gb300" / "csrc" / bench.KERNEL_SOURCES[2][0]
    src.write_text(src.read_text() + "// edited\n")
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) is None


def test_clock_sampler_names_the_gpu_the_rank_runs_on(monkeypatch):
    """nvidia-smi numbers physical GPUs and ignores CUDA_VISIBLE_DEVICES: the
    sampler's selector is the device's UUID, else its PCI bus id, else the
    visible-devices entry of the rank's local index."""
    import torch

    class Props:
        uuid = "1234abcd-0000-1111-2222-333344445555"
        pci_domain_id, pci_bus_id, pci_device_id = 0, 0x1B, 0

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: Props())
    assert bench.gpu_selector(0) == "GPU-1234abcd-0000-1111-2222-333344445555"
    Props.uuid = ""
    assert bench.gpu_selector(0) == "00000000:1B:00.0"

    def unavailable(i):
        raise RuntimeError("no CUDA")

    monkeypatch.setattr(torch.cuda, "get_device_properties", unavailable)
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,7")
    assert bench.gpu_selector(1) == "7"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_selector(2) == "2"
