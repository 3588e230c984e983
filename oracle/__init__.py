"""CPU oracle of the sliding-window GDG decoder: test infrastructure only
(tests/, the smoke check and the CPU legs of bench.py use it; the product
package never does)."""
