"""The benchmark's reference arm on the CPU: the FP64 oracle over a bounded
sample of the default workload prints one JSON line with the keys the
native arm's line has for the workload, the metric and the baseline."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line_on_the_default_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference',
                        '--replicas', '3', '--steps', '1', '--warmup', '1'],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d['impl'] == 'reference'
    assert d['metric'].startswith('tDPD particle-steps/s')
    assert d['unit'] == 'particle-steps/s' and d['higher_is_better'] is True
    assert d['value'] > 0 and d['cpu_baseline']['kind'] == 'oracle' and d['cpu_baseline']['cores'] >= 1
    assert d['config']['name'] == 'ensemble' and d['config']['replicas'] == 3
    assert d['e2e'] == {'value': d['value'], 'unit': d['unit'], 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}
    assert d['steps'] == 1 and d['warmup'] == 1 and d['dtype'] == 'f64'
