"""CPU oracle of the batched rigid-body step (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package. The product library never imports it.
"""
from .oracle import (build, load, step, detect, OracleDetect, cores, loss_and_directional,  # noqa: F401
                     loss_value, step_report, OracleReport, render_depth, step_vjp, OracleVJP, trajectory,
                     goal_seed, rollout_grad, step_f64x, step_lambdas,
                     clip_cap_drops)
