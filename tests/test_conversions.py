"""The integer-pipe float <-> double conversions used where float32 vectors
meet the float64 outer CG agree with the compiler's conversions: every float
bit pattern (float -> double) and edge cases plus 2^26 random doubles
(double -> float, round to nearest even).  Host code only; no GPU needed."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bit_conversions_match_hardware_rounding():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "conv_check")
        subprocess.check_call(["nvcc", "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "conv_check.cu")])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stdout + out.stderr
        assert out.stdout.startswith("OK"), out.stdout
