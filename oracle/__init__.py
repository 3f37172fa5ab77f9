"""FP64 CPU oracle of the rasterizer. Test infrastructure only: the product
package never imports it."""
