"""Host-side pieces of the benchmark that shape its JSON line: the workload sentence
(the same for the GPU arm and the oracle arm), the per-workload training sets of the
learned preconditioner, and the disc size used for point counts (checked against the
oracle's disc)."""
import bench
import oracle as O
import synth


def test_workload_sentence_names_the_benchmark_configuration():
    inp = synth.config_inputs("C3", M=50000, images=False)
    s = bench.workload_name(inp, 6, "learned", "C3")
    assert s == ("N=128 volume, 50000 BF16 128x128 images (60-blob phantom, Haar views, 20 defocus groups, "
                 "SNR 0.05), KB W=6 sigma=2, lambda=1e-3 x Ker(0), learned-preconditioned CG to rel-res 1e-4")
    r = bench.workload_name(synth.config_inputs("RCT", M=10, images=False), 6, "none", "RCT")
    assert "random conical tilt 60 deg" in r and "no CTF" in r and "N=96" in r


def test_training_sets_and_disc_sizes():
    assert bench.TRAIN_DEFAULTS["C3"] == (3000, 96, 10000)
    assert bench.TRAIN_DEFAULTS["C5"] == (2000, 64, 3000)       # as the cap workload's configuration states
    for N in (16, 32, 48, 64, 80, 96, 128):
        assert bench.disc_size(N) == O.disc(N).shape[0]
